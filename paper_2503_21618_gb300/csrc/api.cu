// C ABI of the slrf library: handle lifetime, workspace, and the drivers of
// the hot path (Krylov solve loop, Cholesky-QR2 + Rayleigh-Ritz, Algorithm 1).
#include <cublas_v2.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <climits>
#include <array>
#include <complex>
#include <functional>
#include <future>
#include <map>
#include <memory>
#include <mutex>
#include <type_traits>
#include <string>
#include <thread>
#include <vector>

#include "host_pool.h"
#include "internal.h"
#include "mg.h"
#include "slrf.h"

using namespace slrf;
using cd = std::complex<double>;

namespace {
thread_local std::string g_last_error;

#define CK(call)                                                                        \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess) {                                                        \
            g_last_error = std::string(#call) + ": " + cudaGetErrorString(e_);          \
            return SLRF_ECUDA;                                                          \
        }                                                                               \
    } while (0)
#define CKS(expr)                                   \
    do {                                            \
        slrf_status s_ = (expr);                    \
        if (s_ != SLRF_OK) return s_;               \
    } while (0)

// Pinned, device-mapped host words through which the Krylov loop polls its
// active-column count: one process-wide page handed out in 64-byte slots, so
// creating or destroying a handle never calls cudaHostAlloc/cudaFreeHost
// (which can synchronise the device).
std::mutex g_pin_mu;
int32_t *g_pin_host = nullptr, *g_pin_dev = nullptr;
std::vector<int> g_pin_free;
constexpr int kPinSlots = 1024, kPinStride = 16;

bool pin_acquire(int32_t **hp, int32_t **dp) {
    std::lock_guard<std::mutex> lock(g_pin_mu);
    if (!g_pin_host) {
        if (cudaHostAlloc((void **)&g_pin_host, (size_t)kPinSlots * kPinStride * 4,
                          cudaHostAllocMapped | cudaHostAllocPortable) != cudaSuccess ||
            cudaHostGetDevicePointer((void **)&g_pin_dev, g_pin_host, 0) != cudaSuccess) {
            cudaGetLastError();
            g_pin_host = g_pin_dev = nullptr;
            return false;
        }
        for (int i = kPinSlots - 1; i >= 0; --i) g_pin_free.push_back(i);
    }
    if (g_pin_free.empty()) return false;
    const int i = g_pin_free.back();
    g_pin_free.pop_back();
    *hp = g_pin_host + (size_t)i * kPinStride;
    *dp = g_pin_dev + (size_t)i * kPinStride;
    return true;
}

void pin_release(int32_t *hp) {
    std::lock_guard<std::mutex> lock(g_pin_mu);
    g_pin_free.push_back((int)((hp - g_pin_host) / kPinStride));
}

const char *kKernelClassNames[SLRF_NKERNEL_CLASSES] = {
    "shifted_spmm", "krylov_update", "krylov_direction", "krylov_reduce", "krylov_init", "spmm_real",
    "gram", "tall_gemm", "small_dense", "residual", "filter_combine", "other", "mg_fine", "mg_transfer",
    "mg_coarse"};
}  // namespace

// ---------------------------------------------------------------------------
// Ctx
// ---------------------------------------------------------------------------
namespace slrf {
void Ctx::reset_counters() {
    for (int i = 0; i < SLRF_NKERNEL_CLASSES; ++i) {
        launches[i] = 0;
        bytes[i] = 0;
        flops[i] = 0;
    }
    used = 0;
}
void Ctx::before(int kc, double b, double f) {
    launches[kc] += 1;
    bytes[kc] += b;
    flops[kc] += f;
    rec = profile && ((profile_mask >> kc) & 1u);
    if (rec) {
        if (used == pool.size()) {
            EvPair p;
            cudaEventCreate(&p.a);
            cudaEventCreate(&p.b);
            p.kc = kc;
            pool.push_back(p);
        }
        pool[used].kc = kc;
        cudaEventRecord(pool[used].a, stream);
        cur_kc = kc;
    }
}
void Ctx::after() {
    if (rec) {
        cudaEventRecord(pool[used].b, stream);
        ++used;
    }
    rec = false;
}
void Ctx::harvest(double ms_out[SLRF_NKERNEL_CLASSES]) {
    if (!profile || used == 0) return;
    cudaStreamSynchronize(stream);
    for (size_t i = 0; i < used; ++i) {
        float t = 0;
        if (cudaEventElapsedTime(&t, pool[i].a, pool[i].b) == cudaSuccess) ms_out[pool[i].kc] += t;
    }
    used = 0;
}
void Ctx::destroy() {
    for (auto &p : pool) {
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
    }
    pool.clear();
    used = 0;
}
}  // namespace slrf

// ---------------------------------------------------------------------------
// handle
// ---------------------------------------------------------------------------
struct Buf {
    void *p = nullptr;
    size_t bytes = 0;
};

struct slrf_handle {
    Ctx ctx;
    slrf_opts opts;
    DevPencil A;
    int device = 0;
    size_t pencil_bytes = 0;
    size_t ws_bytes = 0;
    // named workspace buffers (grow only)
    Buf kP, kQ, kR, kDinv, kU, kPart, kSig, kScal, kFlags;
    Buf rOz;   // Ozaki Gram digits and partials
    Buf rOzT;  // Ozaki tall-product digits
    Buf rTallB;   // slrf_tall_product: copy of B
    Buf mgInvPan, mgCtWork;   // exact level on the tensor cores: split inverses, per-apply work
    bool inv_pan_ok = false;
    void *inv_pan_buf = nullptr;
    Buf rW1, rQ1, rQ2, rX, rAX, rBX, rRes, rSmall, rSplit, rV, rTheta, rRho;
    int64_t shifted_cholqr = 0;   // Rayleigh-Ritz steps that needed the shifted fallback
    Buf hostV, hostX;   // device staging for the host-buffer entry points
    // multigrid preconditioner: hierarchy (static), per-solve level blocks, Z
    Buf mgStatic, mgState, kZ;
    Buf kBcg;   // BiCGStab: r^, v, y, z, t blocks and omega scalars
    bool node_blocks = false;             // 3-dof node-block pattern (elasticity)
    bool mg_ready = false;
    // a hierarchy still being built on a host thread when slrf_create
    // returned: waits for it and uploads it (run by the first mg_ensure)
    std::function<slrf_status(slrf_handle *)> mg_finish;
    int mg_block = 0, mg_coarse = 0;      // parameters the hierarchy was built with
    double mg_theta = 0.0;
    // the options' near-null space (n x mg_null_k, copied from the options);
    // mg_null_dirty: set since the hierarchy was built
    std::vector<double> mg_null;
    int mg_null_k = 0;
    bool mg_null_dirty = false;
    std::vector<double> mg_lam;           // coarsest eigenvalues
    // the coarsest level's eigenpairs still being computed on a host thread
    // when the hierarchy was uploaded: waits for them and uploads V (run by
    // the first cycle that reaches the coarsest level)
    std::function<slrf_status(slrf_handle *)> mg_coarse_pending;
    std::vector<int64_t> mg_level_n, mg_level_nnz;
    double mg_setup_ms = 0.0;
    std::vector<char> mg_cinv_host;       // staging of 1/(lambda_k - sigma_j)
    // deep shifts truncate the cycle at the first level where the shift
    // outweighs the diagonal; that level is then solved exactly
    struct MgEig {
        std::vector<double> lam;
        Buf dev;                          // FP32 then FP64 eigenvectors
    } mg_eig[slrf::MG_MAX_LEVELS];
    std::vector<slrf::HostLevel> mg_host_lv;   // level pencils (no transfers)
    std::vector<double> mg_maxba;              // per level max_i b_ii / a_ii
    int mg_nlev_full = 0;
    const float *mg_fullV32 = nullptr;
    const double *mg_fullV64 = nullptr;
    slrf::MgSolve<float> mg32;
    slrf::MgSolve<double> mg64;
    Buf iluPat, iluFac, kIluY;  // ILU preconditioner: pattern (once), factors (per call), sweep scratch
    slrf::IluPattern ilu_pat;
    bool ilu_ready = false;
    Buf mgInv;                  // FP32 cycles: dense shifted inverses of the exact level + their work
    // the poles, level and hierarchy the inverses in mgInv were formed for:
    // the outer steps of one call reuse them instead of inverting again
    std::vector<double> inv_key;
    const void *inv_buf = nullptr;
    int64_t mg_gen = 0;
    cublasHandle_t cublas = nullptr;   // created on first use (coarse-level GEMMs)
    int32_t *h_pin = nullptr;   // pinned host words for polls
    int32_t *d_pin = nullptr;   // device alias of h_pin
    cudaEvent_t ev_poll = nullptr, ev_t0 = nullptr, ev_t1 = nullptr;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> phase_k, phase_r;
    size_t phase_k_used = 0, phase_r_used = 0;
};

namespace {

// Device memory of handles comes from one stream-ordered pool per device,
// created by the library, that keeps what destroyed handles free reserved
// for the next ones: the default pool hands freed memory back to the driver
// at every synchronisation, and mapping it again on the next handle costs
// milliseconds per GB.  slrf_release_cached_memory() trims it.
std::mutex g_pool_mu;
std::map<int, cudaMemPool_t> g_pools;

cudaMemPool_t handle_pool(int device) {
    std::lock_guard<std::mutex> lock(g_pool_mu);
    auto it = g_pools.find(device);
    if (it != g_pools.end()) return it->second;
    cudaMemPool_t pool = nullptr;
    cudaMemPoolProps props;
    memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = device;
    if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
        cudaGetLastError();
        pool = nullptr;   // the device's default pool is used instead
    } else {
        uint64_t keep = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    g_pools[device] = pool;
    return pool;
}

cudaError_t dev_alloc(slrf_handle *h, void **ptr, size_t bytes) {
    cudaMemPool_t pool = handle_pool(h->device);
    return pool ? cudaMallocFromPoolAsync(ptr, bytes, pool, h->ctx.stream) : cudaMallocAsync(ptr, bytes, h->ctx.stream);
}

slrf_status ensure(slrf_handle *h, Buf &b, size_t bytes) {
    if (bytes == 0) bytes = 16;
    if (b.bytes >= bytes) return SLRF_OK;
    if (h->opts.mem_budget > 0 &&
        h->pencil_bytes + h->ws_bytes - b.bytes + bytes > (size_t)h->opts.mem_budget)
        return SLRF_EBUDGET;
    // stream-ordered allocation: growing one handle's workspace never waits
    // for work of other handles on other streams
    if (b.p) {
        cudaFreeAsync(b.p, h->ctx.stream);
        h->ws_bytes -= b.bytes;
        b.p = nullptr;
        b.bytes = 0;
    }
    if (dev_alloc(h, &b.p, bytes) != cudaSuccess) {
        cudaGetLastError();
        b.p = nullptr;
        g_last_error = "device allocation of " + std::to_string(bytes) + " bytes failed";
        return SLRF_ENOMEM;
    }
    b.bytes = bytes;
    h->ws_bytes += bytes;
    return SLRF_OK;
}

template <typename T> T *as(Buf &b) { return reinterpret_cast<T *>(b.p); }

void phase_begin(slrf_handle *h, std::vector<std::pair<cudaEvent_t, cudaEvent_t>> &v, size_t &used) {
    if (used == v.size()) {
        cudaEvent_t a, b;
        cudaEventCreate(&a);
        cudaEventCreate(&b);
        v.push_back({a, b});
    }
    cudaEventRecord(v[used].first, h->ctx.stream);
}
void phase_end(slrf_handle *h, std::vector<std::pair<cudaEvent_t, cudaEvent_t>> &v, size_t &used) {
    cudaEventRecord(v[used].second, h->ctx.stream);
    ++used;
}
double phase_sum(std::vector<std::pair<cudaEvent_t, cudaEvent_t>> &v, size_t &used) {
    double s = 0;
    for (size_t i = 0; i < used; ++i) {
        float t = 0;
        if (cudaEventElapsedTime(&t, v[i].first, v[i].second) == cudaSuccess) s += t;
    }
    used = 0;
    return s;
}

struct CallScope {
    slrf_handle *h;
    slrf_report *rep;
    explicit CallScope(slrf_handle *h_, slrf_report *r) : h(h_), rep(r) {
        // every call forms its own exact-level inverses (reused by its outer steps only)
        h->inv_key.clear();
        h->ctx.reset_counters();
        h->phase_k_used = h->phase_r_used = 0;
        cudaEventRecord(h->ev_t0, h->ctx.stream);
        if (rep) memset(rep, 0, sizeof(*rep));
    }
    void finish() {
        cudaEventRecord(h->ev_t1, h->ctx.stream);
        cudaEventSynchronize(h->ev_t1);
        if (!rep) {
            h->ctx.used = 0;
            h->phase_k_used = h->phase_r_used = 0;
            return;
        }
        float t = 0;
        cudaEventElapsedTime(&t, h->ev_t0, h->ev_t1);
        rep->ms_total = t;
        rep->ms_krylov = phase_sum(h->phase_k, h->phase_k_used);
        rep->ms_rr = phase_sum(h->phase_r, h->phase_r_used);
        int64_t tot = 0;
        for (int i = 0; i < SLRF_NKERNEL_CLASSES; ++i) {
            rep->k_launches[i] = h->ctx.launches[i];
            rep->k_bytes[i] = h->ctx.bytes[i];
            rep->k_flops[i] = h->ctx.flops[i];
            tot += h->ctx.launches[i];
        }
        rep->kernel_launches = tot;
        h->ctx.harvest(rep->k_ms);
    }
};

slrf_status check_filter(const slrf_filter *f) {
    if (!f || f->n_poles < 1 || f->n_poles > SLRF_MAX_POLES || !f->sigma_re || !f->sigma_im || !f->w_re ||
        !f->w_im)
        return SLRF_EINVAL;
    for (int j = 0; j < f->n_poles; ++j) {
        if (!isfinite(f->sigma_re[j]) || !isfinite(f->sigma_im[j]) || !isfinite(f->w_re[j]) ||
            !isfinite(f->w_im[j]) || f->sigma_im[j] == 0.0)
            return SLRF_EINVAL;
    }
    return SLRF_OK;
}

template <typename T> PoleSet<T> make_poleset(const slrf_filter *f) {
    PoleSet<T> ps;
    ps.N = f->n_poles;
    for (int j = 0; j < SLRF_MAX_POLES; ++j) {
        ps.re[j] = j < f->n_poles ? (T)f->sigma_re[j] : (T)0;
        ps.im[j] = j < f->n_poles ? (T)f->sigma_im[j] : (T)0;
    }
    return ps;
}

// ----- pencil setup kernels ------------------------------------------------
__global__ void k_pack_ab(int64_t nnz, const double *a, const double *b, float2 *ab32, double2 *ab64) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= nnz) return;
    ab32[k] = make_float2((float)a[k], (float)b[k]);
    ab64[k] = make_double2(a[k], b[k]);
}
__global__ void k_diag(int n, const int32_t *rowptr, const int32_t *col, const double *a, const double *b,
                       double *da, double *db) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double x = 0, y = 0;
    for (int k = rowptr[i]; k < rowptr[i + 1]; ++k)
        if (col[k] == i) {
            x = a[k];
            y = b[k];
        }
    da[i] = x;
    db[i] = y;
}
// Row-group form on the device, from the uploaded CSR (rows sorted by
// column): group g holds rows gR .. gR+R-1; its entries are the union of
// their columns, ascending, with R (a, b) pairs per entry (zeros where a row
// has no entry, and for the rows past n of a ragged last group).  Each
// thread merges the R rows of one group: once to count (into gptr[g + 1]),
// and after the prefix sum to write.
__device__ __forceinline__ int rg_next(int R, const int32_t *col, const int *p, const int *e) {
    int c = INT_MAX;
    for (int r = 0; r < R; ++r)
        if (p[r] < e[r]) c = min(c, col[p[r]]);
    return c;
}
__global__ void k_rg_count(int64_t n, int R, int64_t ng, const int32_t *rowptr, const int32_t *col, int32_t *gptr) {
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= ng) return;
    int p[4], e[4];
    for (int r = 0; r < R; ++r) {
        const int64_t row = g * R + r;
        p[r] = row < n ? rowptr[row] : 0;
        e[r] = row < n ? rowptr[row + 1] : 0;
    }
    int cnt = 0;
    for (int c = rg_next(R, col, p, e); c != INT_MAX; c = rg_next(R, col, p, e), ++cnt)
        for (int r = 0; r < R; ++r)
            if (p[r] < e[r] && col[p[r]] == c) ++p[r];
    gptr[g + 1] = cnt;
    if (g == 0) gptr[0] = 0;
}
// In-place inclusive prefix sum of gptr[1 .. ng] (one block of 1024 threads,
// each over a contiguous chunk) and the largest group size in *emax.
__global__ void __launch_bounds__(1024) k_rg_scan(int64_t ng, int32_t *gptr, int32_t *emax) {
    __shared__ int64_t part[1024];
    __shared__ int32_t mx[1024];
    const int t = threadIdx.x;
    const int64_t c0 = 1 + ng * t / 1024, c1 = 1 + ng * (t + 1) / 1024;
    int64_t sum = 0;
    int32_t m = 0;
    for (int64_t i = c0; i < c1; ++i) {
        sum += gptr[i];
        m = max(m, gptr[i]);
    }
    part[t] = sum;
    mx[t] = m;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {   // Hillis-Steele over the chunk sums
        const int64_t v = t >= off ? part[t - off] : 0;
        const int32_t w = t >= off ? mx[t - off] : 0;
        __syncthreads();
        part[t] += v;
        mx[t] = max(mx[t], w);
        __syncthreads();
    }
    int64_t run = t ? part[t - 1] : 0;
    for (int64_t i = c0; i < c1; ++i) {
        run += gptr[i];
        gptr[i] = (int32_t)run;
    }
    if (t == 1023) *emax = mx[1023];
}
__global__ void k_rg_fill(int64_t n, int R, int64_t ng, const int32_t *rowptr, const int32_t *col, const double *a,
                          const double *b, const int32_t *gptr, int32_t *ucol, float2 *ab32, double2 *ab64,
                          float4 *ab4, uint8_t *dpos) {
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= ng) return;
    int p[4], e[4];
    for (int r = 0; r < R; ++r) {
        const int64_t row = g * R + r;
        p[r] = row < n ? rowptr[row] : 0;
        e[r] = row < n ? rowptr[row + 1] : 0;
        if (dpos) dpos[g * R + r] = 0;
    }
    const int64_t o0 = gptr[g];
    int64_t o = o0;
    for (int c = rg_next(R, col, p, e); c != INT_MAX; c = rg_next(R, col, p, e), ++o) {
        ucol[o] = c;
        for (int r = 0; r < R; ++r) {
            double x = 0.0, y = 0.0;
            if (p[r] < e[r] && col[p[r]] == c) {
                x = a[p[r]];
                y = b[p[r]];
                ++p[r];
            }
            const int64_t q = o * R + r;
            ab64[q] = make_double2(x, y);
            ab32[q] = make_float2((float)x, (float)y);
            if (ab4) ab4[q] = make_float4((float)x, (float)x, (float)y, (float)y);
            if (dpos && c == g * R + r) dpos[g * R + r] = (uint8_t)(o - o0);
        }
    }
}
__global__ void k_symmetrize(int m, double *S) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= (int64_t)m * m) return;
    const int i = (int)(e / m), j = (int)(e % m);
    if (j <= i) return;
    const double v = 0.5 * (S[(int64_t)i * m + j] + S[(int64_t)j * m + i]);
    S[(int64_t)i * m + j] = v;
    S[(int64_t)j * m + i] = v;
}

// ---------------------------------------------------------------------------
// row-group form of the pencil for the shifted SpMM
// ---------------------------------------------------------------------------
bool has_node_blocks(int64_t n, const std::vector<int32_t> &rp, const std::vector<int32_t> &ci, int R) {
    if (n % R) return false;
    for (int64_t g = 0; g < n / R; ++g) {
        const int64_t r0 = g * R;
        const int64_t len = rp[r0 + 1] - rp[r0];
        for (int r = 1; r < R; ++r) {
            if (rp[r0 + r + 1] - rp[r0 + r] != len) return false;
            if (!std::equal(ci.begin() + rp[r0], ci.begin() + rp[r0 + 1], ci.begin() + rp[r0 + r])) return false;
        }
    }
    return true;
}

// Node-block form of a 3-dof pencil (rows of a node share one pattern, made
// of whole neighbour nodes, and the mass couples equal dofs only): per node
// the neighbour nodes and, per neighbour, the 3 x 3 stiffness block and the 3
// mass weights in three float4.  False (nothing built) when the pencil is
// not of that form.
bool build_nodeblocks(int64_t n, const std::vector<int32_t> &rp, const std::vector<int32_t> &ci,
                      const std::vector<double> &av, const std::vector<double> &bv, std::vector<int32_t> &nptr,
                      std::vector<int32_t> &nnode, std::vector<float4> &coef) {
    if (n % 3 || !has_node_blocks(n, rp, ci, 3)) return false;
    const int64_t nn = n / 3;
    nptr.assign(nn + 1, 0);
    nnode.clear();
    coef.clear();
    for (int64_t g = 0; g < nn; ++g) {
        const int64_t k0 = rp[3 * g], k1 = rp[3 * g + 1];
        if ((k1 - k0) % 3) return false;
        for (int64_t k = k0; k < k1; k += 3) {
            if (ci[k] % 3 || ci[k + 1] != ci[k] + 1 || ci[k + 2] != ci[k] + 2) return false;
            float a[3][3], b[3];
            for (int r = 0; r < 3; ++r) {
                const int64_t kr = rp[3 * g + r] + (k - k0);
                for (int c = 0; c < 3; ++c) {
                    a[r][c] = (float)av[kr + c];
                    if (c == r) b[r] = (float)bv[kr + c];
                    else if (bv[kr + c] != 0.0) return false;
                }
            }
            nnode.push_back(ci[k] / 3);
            coef.push_back(make_float4(a[0][0], a[0][1], a[0][2], a[1][0]));
            coef.push_back(make_float4(a[1][1], a[1][2], a[2][0], a[2][1]));
            coef.push_back(make_float4(a[2][2], b[0], b[1], b[2]));
        }
        nptr[g + 1] = (int32_t)nnode.size();
    }
    return true;
}

// SELL-C-sigma form of the pencil (FP32 pairs): rows sorted by length,
// longest first, within windows of sigma rows (stable, so equal lengths keep
// their order), chunks of C permuted rows, each padded to its longest row and
// stored slot-major.  Padding slots hold the row's own column and zero
// coefficients.
bool build_sell(int64_t n, const std::vector<int32_t> &rp, const std::vector<int32_t> &ci,
                const std::vector<double> &av, const std::vector<double> &bv, int C, int sigma,
                std::vector<int32_t> &cptr, std::vector<int32_t> &col, std::vector<float2> &ab,
                std::vector<int32_t> &perm, std::vector<int32_t> &rlen) {
    perm.resize(n);
    for (int64_t i = 0; i < n; ++i) perm[i] = (int32_t)i;
    auto len = [&](int32_t r) { return rp[r + 1] - rp[r]; };
    for (int64_t w0 = 0; w0 < n; w0 += sigma)
        std::stable_sort(perm.begin() + w0, perm.begin() + std::min<int64_t>(n, w0 + sigma),
                         [&](int32_t x, int32_t y) { return len(x) > len(y); });
    rlen.resize(n);
    for (int64_t i = 0; i < n; ++i) rlen[i] = len(perm[i]);
    const int64_t nch = (n + C - 1) / C;
    cptr.assign(nch + 1, 0);
    int64_t tot = 0;
    for (int64_t c = 0; c < nch; ++c) {
        int32_t K = 0;
        for (int64_t r = c * C; r < std::min<int64_t>(n, (c + 1) * C); ++r) K = std::max(K, rlen[r]);
        tot += (int64_t)K * C;
        if (tot > (1LL << 31) - 1) return false;   // slots addressed by int32 offsets
        cptr[c + 1] = (int32_t)tot;
    }
    col.assign(cptr[nch], 0);
    ab.assign(cptr[nch], make_float2(0.f, 0.f));
    for (int64_t c = 0; c < nch; ++c) {
        const int32_t K = (cptr[c + 1] - cptr[c]) / C;
        for (int r = 0; r < C; ++r) {
            const int64_t pr = c * C + r;
            const int32_t row = pr < n ? perm[pr] : 0;
            for (int32_t k = 0; k < K; ++k) {
                const int64_t e = cptr[c] + (int64_t)k * C + r;
                if (pr < n && k < rlen[pr]) {
                    const int64_t src = rp[row] + k;
                    col[e] = ci[src];
                    ab[e] = make_float2((float)av[src], (float)bv[src]);
                } else {
                    col[e] = row;
                }
            }
        }
    }
    return true;
}

// CSR monotone with sorted, in-range columns, finite values and a positive
// diagonal in every row (SPD pencils have one).
bool pencil_valid(int64_t n, int64_t nnz, const std::vector<int32_t> &rp, const std::vector<int32_t> &ci,
                  const std::vector<double> &av, const std::vector<double> &bv) {
    if (rp[0] != 0 || rp[n] != nnz) return false;
    for (int64_t i = 0; i < n; ++i)
        if (rp[i + 1] < rp[i]) return false;
    // rows in parallel: columns in range and strictly increasing, values
    // finite, a positive diagonal in A and B
    std::atomic<bool> ok{true};
    host_parallel_rows((int)n, host_threads(nnz), [&](int r0, int r1, int) {
        for (int64_t i = r0; i < r1; ++i) {
            bool diag = false;
            for (int64_t k = rp[i]; k < rp[i + 1]; ++k) {
                if (ci[k] < 0 || ci[k] >= n || (k > rp[i] && ci[k] <= ci[k - 1]) || !isfinite(av[k]) ||
                    !isfinite(bv[k])) {
                    ok.store(false, std::memory_order_relaxed);
                    return;
                }
                if (ci[k] == i) diag = av[k] > 0 && bv[k] > 0;
            }
            if (!diag) {
                ok.store(false, std::memory_order_relaxed);
                return;
            }
        }
    });
    return ok.load();
}

// ---------------------------------------------------------------------------
// multigrid hierarchy: host build, upload, per-solve preparation
// ---------------------------------------------------------------------------
int mg_block_for(const slrf_opts &o, int64_t n, const std::vector<int32_t> &rp, const std::vector<int32_t> &ci) {
    if (o.mg_block > 0) return o.mg_block;
    return has_node_blocks(n, rp, ci, 3) ? 3 : 1;
}

// The options' near-null space (n x mg_n_null, host), copied; false if an
// entry is not finite.  Empty when mg_n_null is 0.
bool copy_near_null(const slrf_opts &o, int64_t n, std::vector<double> &out) {
    out.clear();
    if (o.mg_n_null <= 0) return true;
    out.assign(o.mg_near_null, o.mg_near_null + (size_t)n * o.mg_n_null);
    for (double v : out)
        if (!isfinite(v)) return false;
    return true;
}

MgParams mg_params(const slrf_opts &o, int block) {
    MgParams prm;
    prm.block = block;
    prm.coarse_target = o.mg_coarse;
    prm.max_levels = MG_MAX_LEVELS;
    prm.theta = o.mg_theta > 0 ? o.mg_theta : 0.08;
    return prm;
}

// Pack the hierarchy into one device buffer: level pencils (levels
// 1 .. nlev-2; the coarsest is solved exactly), transfers P and P^T (FP32 and
// FP64 values), coarsest eigenvectors (FP32 and FP64).
// Device image of a host hierarchy, laid out and filled on the host (the
// setup thread does this while the pencil uploads): byte offsets of every
// array in one buffer.
struct MgLvOff {
    size_t ptr = 0, col = 0, ab32 = 0, ab64 = 0, da = 0, db = 0;
    size_t pptr = 0, pcol = 0, pv32 = 0, pv64 = 0, rptr = 0, rcol = 0, rv32 = 0, rv64 = 0;
};
struct MgStaged {
    std::unique_ptr<char[]> stage;   // the uploaded part of the image (uninitialised padding)
    size_t upload_bytes = 0, total_bytes = 0;
    std::vector<MgLvOff> lo;
    size_t v32 = 0, v64 = 0, o_fup = 0, o_fuc = 0, o_fdp = 0, o_fdc = 0, o_fq = 0, o_fab32 = 0, o_fab64 = 0;
    int64_t fu_nnz = 0, fd_nnz = 0;
};

// Lays out and fills the image of every level but the coarsest level's
// eigenvectors (mg_stage_v, once they exist).  R0: rows per group of the
// finest level's row-group form (1 = plain rows).  The folded pairs f_ab
// come last and are not uploaded: every solve writes them from f_q.
void mg_stage(const HostHierarchy &H, int R0, MgStaged &S) {
    const int nlev = (int)H.lv.size();
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += (bytes + 255) / 256 * 256;
        return o;
    };
    std::vector<MgLvOff> &lo = S.lo;
    lo.assign(nlev, MgLvOff());
    for (int l = 0; l < nlev; ++l) {
        const HostLevel &L = H.lv[l];
        if (l >= 1 && l < nlev - 1) {
            const size_t nz = L.col.size();
            lo[l].ptr = take((L.n + 1) * 4);
            lo[l].col = take(nz * 4);
            lo[l].ab32 = take(nz * 8);
            lo[l].ab64 = take(nz * 16);
            lo[l].da = take(L.n * 8);
            lo[l].db = take(L.n * 8);
        }
        if (l < nlev - 1) {
            const size_t pz = L.P.col.size();
            lo[l].pptr = take((L.P.n_rows + 1) * 4);
            lo[l].pcol = take(pz * 4);
            lo[l].pv32 = take(pz * 4);
            lo[l].pv64 = take(pz * 8);
            lo[l].rptr = take((L.Rt.n_rows + 1) * 4);
            lo[l].rcol = take(pz * 4);
            lo[l].rv32 = take(pz * 4);
            lo[l].rv64 = take(pz * 8);
        }
    }
    const int nc = H.lv.back().n;
    S.v32 = take((size_t)nc * nc * 4);
    S.v64 = take((size_t)nc * nc * 8);
    // fused finest-level transfers: F by fine row groups ("up") and by coarse rows ("down")
    FusedLayout FL;
    if (nlev > 1) mg_fused_pattern(H.lv[0], H.lv[1].n, R0, FL);
    const size_t nq = nlev > 1 ? FL.q_count() : 0;
    const size_t nslot = nq / 4;   // 4 doubles = two double2 per stored pair
    S.o_fup = take(FL.up_ptr.size() * 4);
    S.o_fuc = take(FL.up_col.size() * 4);
    S.o_fdp = take(FL.down_ptr.size() * 4);
    S.o_fdc = take(FL.down_col.size() * 4);
    S.o_fq = take(nq * sizeof(double));
    S.upload_bytes = off;
    S.o_fab32 = take(nslot * sizeof(float2));
    S.o_fab64 = take(nslot * sizeof(double2));
    S.total_bytes = off;
    S.fu_nnz = (int64_t)FL.up_col.size();
    S.fd_nnz = (int64_t)FL.down_col.size();
    S.stage.reset(new char[S.upload_bytes]);
    char *stage = S.stage.get();
    auto put = [&](size_t o, const void *src, size_t bytes) {
        if (bytes) memcpy(stage + o, src, bytes);
    };
    for (int l = 0; l < nlev; ++l) {
        const HostLevel &L = H.lv[l];
        if (l >= 1 && l < nlev - 1) {
            const size_t nz = L.col.size();
            put(lo[l].ptr, L.ptr.data(), (L.n + 1) * 4);
            put(lo[l].col, L.col.data(), nz * 4);
            float2 *a32 = reinterpret_cast<float2 *>(stage + lo[l].ab32);
            double2 *a64 = reinterpret_cast<double2 *>(stage + lo[l].ab64);
            for (size_t k = 0; k < nz; ++k) {
                a32[k] = make_float2((float)L.a[k], (float)L.b[k]);
                a64[k] = make_double2(L.a[k], L.b[k]);
            }
            put(lo[l].da, L.diag_a.data(), L.n * 8);
            put(lo[l].db, L.diag_b.data(), L.n * 8);
        }
        if (l < nlev - 1) {
            const size_t pz = L.P.col.size();
            put(lo[l].pptr, L.P.ptr.data(), (L.P.n_rows + 1) * 4);
            put(lo[l].pcol, L.P.col.data(), pz * 4);
            put(lo[l].pv64, L.P.val.data(), pz * 8);
            put(lo[l].rptr, L.Rt.ptr.data(), (L.Rt.n_rows + 1) * 4);
            put(lo[l].rcol, L.Rt.col.data(), pz * 4);
            put(lo[l].rv64, L.Rt.val.data(), pz * 8);
            float *p32 = reinterpret_cast<float *>(stage + lo[l].pv32);
            float *r32 = reinterpret_cast<float *>(stage + lo[l].rv32);
            for (size_t k = 0; k < pz; ++k) {
                p32[k] = (float)L.P.val[k];
                r32[k] = (float)L.Rt.val[k];
            }
        }
    }
    put(S.o_fup, FL.up_ptr.data(), FL.up_ptr.size() * 4);
    put(S.o_fuc, FL.up_col.data(), FL.up_col.size() * 4);
    put(S.o_fdp, FL.down_ptr.data(), FL.down_ptr.size() * 4);
    put(S.o_fdc, FL.down_col.data(), FL.down_col.size() * 4);
    if (nq) mg_fused_values(H.lv[0], FL, reinterpret_cast<double *>(stage + S.o_fq));
}

void mg_stage_v(const HostHierarchy &H, MgStaged &S) {
    const size_t nc = (size_t)H.lv.back().n;
    float *V32 = reinterpret_cast<float *>(S.stage.get() + S.v32);
    for (size_t k = 0; k < nc * nc; ++k) V32[k] = (float)H.V[k];
    memcpy(S.stage.get() + S.v64, H.V.data(), nc * nc * 8);
}

// Hp / eig: the hierarchy (kept alive) whose coarsest eigenpairs a host
// thread is still computing; H.lam and the staged V are then not read.
slrf_status mg_upload(slrf_handle *h, const HostHierarchy &H, const MgStaged &S, int block,
                      std::shared_ptr<HostHierarchy> Hp = nullptr, std::shared_future<std::string> eig = {}) {
    const int nlev = (int)H.lv.size();
    if (nlev > MG_MAX_LEVELS) {
        g_last_error = "multigrid setup: too many levels";
        return SLRF_BREAKDOWN;
    }
    const int nc = H.lv.back().n;
    const std::vector<MgLvOff> &lo = S.lo;
    CKS(ensure(h, h->mgStatic, S.total_bytes));
    char *base = reinterpret_cast<char *>(h->mgStatic.p);
    CK(cudaMemcpyAsync(base, S.stage.get(), S.upload_bytes, cudaMemcpyHostToDevice, h->ctx.stream));
    CK(cudaStreamSynchronize(h->ctx.stream));   // the staging vector is pageable
    auto fill = [&](auto &mg, auto tag) {
        using T = decltype(tag);
        mg = std::remove_reference_t<decltype(mg)>();
        mg.nlev = nlev;
        mg.nc = nc;
        const DevPencil &A = h->A;
        MgLevel<T> &L0 = mg.lv[0];
        L0.R = A.rg_rows > 1 ? A.rg_rows : 1;
        L0.ngroups = A.rg_rows > 1 ? A.rg_ngroups : A.n;
        L0.nnz_union = A.rg_rows > 1 ? A.rg_nnz : A.nnz;
        L0.gptr = A.rg_rows > 1 ? A.rg_ptr : A.rowptr;
        L0.gcol = A.rg_rows > 1 ? A.rg_col : A.col;
        if (sizeof(T) == 4)
            L0.ab = reinterpret_cast<const cplx<T> *>(A.rg_rows > 1 ? (const void *)A.rg_ab32 : (const void *)A.ab32);
        else
            L0.ab = reinterpret_cast<const cplx<T> *>(A.rg_rows > 1 ? (const void *)A.rg_ab64 : (const void *)A.ab64);
        L0.diag_a = A.diag_a;
        L0.diag_b = A.diag_b;
        for (int l = 0; l < nlev; ++l) {
            const HostLevel &HL = H.lv[l];
            MgLevel<T> &L = mg.lv[l];
            L.n = HL.n;
            L.rho = HL.rho;
            if (l >= 1 && l < nlev - 1) {
                L.R = 1;
                L.ngroups = HL.n;
                L.nnz_union = (int64_t)HL.col.size();
                L.gptr = reinterpret_cast<const int32_t *>(base + lo[l].ptr);
                L.gcol = reinterpret_cast<const int32_t *>(base + lo[l].col);
                L.ab = reinterpret_cast<const cplx<T> *>(base + (sizeof(T) == 4 ? lo[l].ab32 : lo[l].ab64));
                L.diag_a = reinterpret_cast<const double *>(base + lo[l].da);
                L.diag_b = reinterpret_cast<const double *>(base + lo[l].db);
            }
            if (l < nlev - 1) {
                L.p_nnz = L.r_nnz = (int64_t)HL.P.col.size();
                L.pptr = reinterpret_cast<const int32_t *>(base + lo[l].pptr);
                L.pcol = reinterpret_cast<const int32_t *>(base + lo[l].pcol);
                L.pval = reinterpret_cast<const T *>(base + (sizeof(T) == 4 ? lo[l].pv32 : lo[l].pv64));
                L.rptr = reinterpret_cast<const int32_t *>(base + lo[l].rptr);
                L.rcol = reinterpret_cast<const int32_t *>(base + lo[l].rcol);
                L.rval = reinterpret_cast<const T *>(base + (sizeof(T) == 4 ? lo[l].rv32 : lo[l].rv64));
            }
        }
        mg.V = reinterpret_cast<const T *>(base + (sizeof(T) == 4 ? S.v32 : S.v64));
        if (nlev > 1) {
            L0.fu_nnz = S.fu_nnz;
            L0.fd_nnz = S.fd_nnz;
            L0.fu_ptr = reinterpret_cast<const int32_t *>(base + S.o_fup);
            L0.fu_col = reinterpret_cast<const int32_t *>(base + S.o_fuc);
            L0.fd_ptr = reinterpret_cast<const int32_t *>(base + S.o_fdp);
            L0.fd_col = reinterpret_cast<const int32_t *>(base + S.o_fdc);
            L0.f_q = reinterpret_cast<const double2 *>(base + S.o_fq);
            L0.f_ab = reinterpret_cast<cplx<T> *>(base + (sizeof(T) == 4 ? S.o_fab32 : S.o_fab64));
        }
    };
    fill(h->mg32, 0.0f);
    fill(h->mg64, 0.0);
    h->mg_nlev_full = nlev;
    h->mg_fullV32 = h->mg32.V;
    h->mg_fullV64 = h->mg64.V;
    h->mg_coarse_pending = nullptr;
    if (eig.valid() && Hp) {
        h->mg_lam.clear();
        float *v32 = const_cast<float *>(h->mg_fullV32);
        double *v64 = const_cast<double *>(h->mg_fullV64);
        h->mg_coarse_pending = [Hp, eig, v32, v64](slrf_handle *hh) -> slrf_status {
            std::string err;
            try {
                err = eig.get();
            } catch (const std::exception &ex) {
                err = std::string("multigrid setup: ") + ex.what();
            }
            if (!err.empty()) {
                g_last_error = err;
                return SLRF_BREAKDOWN;
            }
            const size_t nn = Hp->V.size();
            std::vector<float> V32(nn);
            for (size_t k = 0; k < nn; ++k) V32[k] = (float)Hp->V[k];
            CK(cudaMemcpyAsync(v32, V32.data(), nn * 4, cudaMemcpyHostToDevice, hh->ctx.stream));
            CK(cudaMemcpyAsync(v64, Hp->V.data(), nn * 8, cudaMemcpyHostToDevice, hh->ctx.stream));
            CK(cudaStreamSynchronize(hh->ctx.stream));   // pageable sources
            hh->mg_lam = Hp->lam;
            return SLRF_OK;
        };
    } else {
        h->mg_lam = H.lam;
    }
    h->mg_maxba.clear();
    h->mg_host_lv.clear();
    for (int l = 0; l < nlev; ++l) {
        h->mg_maxba.push_back(H.lv[l].maxba);
        HostLevel c;
        c.n = H.lv[l].n;
        if (l >= 1) {
            c.ptr = H.lv[l].ptr;
            c.col = H.lv[l].col;
            c.a = H.lv[l].a;
            c.b = H.lv[l].b;
        }
        h->mg_host_lv.push_back(std::move(c));
    }
    for (auto &e : h->mg_eig) e.lam.clear();
    h->mg_level_n.clear();
    h->mg_level_nnz.clear();
    for (int l = 0; l < nlev; ++l) {
        h->mg_level_n.push_back(H.lv[l].n);
        h->mg_level_nnz.push_back(l == 0 ? h->A.nnz : (int64_t)H.lv[l].col.size());
    }
    h->mg_setup_ms = H.ms_setup;
    h->mg_block = block;
    h->mg_coarse = h->opts.mg_coarse;
    h->mg_theta = h->opts.mg_theta;
    h->mg_ready = true;
    ++h->mg_gen;
    return SLRF_OK;
}

slrf_status mg_build_upload(slrf_handle *h, const std::vector<int32_t> &rp, const std::vector<int32_t> &ci,
                            const std::vector<double> &av, const std::vector<double> &bv) {
    const int block = mg_block_for(h->opts, h->A.n, rp, ci);
    MgParams prm = mg_params(h->opts, block);
    prm.near_null = h->mg_null_k ? h->mg_null.data() : nullptr;
    prm.n_null = h->mg_null_k;
    HostHierarchy H;
    const std::string err = mg_build(h->A.n, rp.data(), ci.data(), av.data(), bv.data(), prm, H);
    if (!err.empty()) {
        g_last_error = err;
        return SLRF_BREAKDOWN;
    }
    MgStaged S;
    mg_stage(H, h->A.rg_rows > 1 ? h->A.rg_rows : 1, S);
    mg_stage_v(H, S);
    CKS(mg_upload(h, H, S, block));
    h->mg_null_dirty = false;
    return SLRF_OK;
}

// Build the hierarchy if the options ask for one it does not have yet (from
// the device copy of the pencil).
slrf_status mg_ensure(slrf_handle *h) {
    if (h->mg_finish) {   // the setup thread of slrf_create
        auto fin = std::move(h->mg_finish);
        h->mg_finish = nullptr;
        CKS(fin(h));
    }
    if (h->mg_ready && h->mg_coarse == h->opts.mg_coarse && h->mg_theta == h->opts.mg_theta &&
        (h->opts.mg_block == 0 || h->opts.mg_block == h->mg_block) && !h->mg_null_dirty)
        return SLRF_OK;
    const int64_t n = h->A.n, nnz = h->A.nnz;
    std::vector<int32_t> rp(n + 1), ci(nnz);
    std::vector<double> av(nnz), bv(nnz);
    CK(cudaMemcpyAsync(rp.data(), h->A.rowptr, (n + 1) * 4, cudaMemcpyDeviceToHost, h->ctx.stream));
    CK(cudaMemcpyAsync(ci.data(), h->A.col, nnz * 4, cudaMemcpyDeviceToHost, h->ctx.stream));
    CK(cudaMemcpyAsync(av.data(), h->A.a, nnz * 8, cudaMemcpyDeviceToHost, h->ctx.stream));
    CK(cudaMemcpyAsync(bv.data(), h->A.b, nnz * 8, cudaMemcpyDeviceToHost, h->ctx.stream));
    CK(cudaStreamSynchronize(h->ctx.stream));
    return mg_build_upload(h, rp, ci, av, bv);
}

// SLRF_PRECOND_AUTO: multigrid for scalar pencils; Jacobi for 3-dof
// node-block (elasticity) pencils, where the translation-only aggregation
// of the hierarchy measured no faster than Jacobi on shifts deep inside
// the spectrum.
bool uses_mg(const slrf_handle *h) {
    return h->opts.precond == SLRF_PRECOND_MG || (h->opts.precond == SLRF_PRECOND_AUTO && !h->node_blocks);
}

template <typename T> MgSolve<T> &mg_of(slrf_handle *h);
template <> MgSolve<float> &mg_of<float>(slrf_handle *h) { return h->mg32; }
template <> MgSolve<double> &mg_of<double>(slrf_handle *h) { return h->mg64; }

constexpr int kMgExactMax = 768;   // largest level diagonalised on demand (host, O(n^3))

// Per-solve level blocks, 1/(lambda_k - sigma_j) and the damped Jacobi
// diagonals of every smoothed level.  The cycle stops at the first level
// whose shift weight max_j |sigma_j| max_i b_ii/a_ii exceeds mg_shift_limit
// (there a Jacobi sweep no longer smooths the shifted operator); that level
// is solved exactly.  *usable = false (AUTO only) when that level is too
// large to diagonalise: the caller then uses Jacobi for this solve.
template <typename T>
slrf_status mg_prepare(slrf_handle *h, const slrf_filter *f, const KrylovDims &d, KrylovBuffers<T> &kb,
                       bool allow_fallback, bool *usable) {
    *usable = true;
    CKS(mg_ensure(h));
    MgSolve<T> &mg = mg_of<T>(h);
    const int nfull = h->mg_nlev_full;
    double smax = 0.0;
    for (int j = 0; j < f->n_poles; ++j) smax = std::max(smax, std::hypot(f->sigma_re[j], f->sigma_im[j]));
    int c = nfull - 1;
    for (int l = 1; l < nfull - 1; ++l)
        if (smax * h->mg_maxba[l] > h->opts.mg_shift_limit) {
            c = l;
            break;
        }
    // FP32 cycles: the first level below the finest (not the coarsest) with
    // at most mg_exact unknowns ends the cycle with its dense shifted inverses
    int e_inv = -1;
    if (sizeof(T) == 4 && h->opts.mg_exact > 0)
        for (int l = 1; l <= c && l < nfull - 1; ++l)
            if (h->mg_host_lv[l].n <= h->opts.mg_exact) {
                e_inv = l;
                break;
            }
    if (e_inv >= 0) c = e_inv;
    const std::vector<double> *lam = &h->mg_lam;
    const T *V = reinterpret_cast<const T *>(sizeof(T) == 4 ? (const void *)h->mg_fullV32 : (const void *)h->mg_fullV64);
    if (e_inv < 0 && c < nfull - 1) {
        auto &E = h->mg_eig[c];
        const int ncl = h->mg_host_lv[c].n;
        if (E.lam.empty() && ncl > kMgExactMax) {
            if (allow_fallback) {
                *usable = false;
                return SLRF_OK;
            }
            c = nfull - 1;   // explicit MG: keep the full cycle
        } else {
            if (E.lam.empty()) {
                std::vector<double> Vh;
                const std::string err = mg_level_eig(h->mg_host_lv[c], Vh, E.lam);
                if (!err.empty()) {
                    E.lam.clear();
                    g_last_error = err;
                    return SLRF_BREAKDOWN;
                }
                const size_t nn = (size_t)ncl * ncl;
                const size_t off64 = (nn * 4 + 255) / 256 * 256;
                CKS(ensure(h, E.dev, off64 + nn * 8));
                std::vector<char> stage(off64 + nn * 8);
                float *v32 = reinterpret_cast<float *>(stage.data());
                for (size_t k = 0; k < nn; ++k) v32[k] = (float)Vh[k];
                memcpy(stage.data() + off64, Vh.data(), nn * 8);
                CK(cudaMemcpyAsync(E.dev.p, stage.data(), stage.size(), cudaMemcpyHostToDevice, h->ctx.stream));
                CK(cudaStreamSynchronize(h->ctx.stream));   // pageable staging
            }
            const size_t off64 = ((size_t)ncl * ncl * 4 + 255) / 256 * 256;
            V = reinterpret_cast<const T *>(reinterpret_cast<char *>(E.dev.p) + (sizeof(T) == 4 ? 0 : off64));
            lam = &E.lam;
        }
    }
    if (e_inv < 0 && c == nfull - 1 && h->mg_coarse_pending) {   // the cycle reaches the coarsest level
        CKS(h->mg_coarse_pending(h));
        h->mg_coarse_pending = nullptr;
    }
    mg.nlev = c + 1;
    mg.nc = h->mg_host_lv[c].n;
    mg.V = V;
    // auto (0): one sweep per side when the cycle ends at the exact level
    // (measured on the 2D workload: 224 against 230 ms per solve with two,
    // 10.4 against 10.2 iterations per pole), else two
    mg.nu = h->opts.mg_nu > 0 ? h->opts.mg_nu : (e_inv >= 0 ? 1 : 2);
    mg.gamma = std::max(1, h->opts.mg_cycle);
    mg.omega = h->opts.mg_omega;
    const int W = d.W(), N = d.N, nc = mg.nc;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += (bytes + 255) / 256 * 256;
        return o;
    };
    std::vector<size_t> o_r(mg.nlev), o_z(mg.nlev), o_t(mg.nlev), o_d(mg.nlev);
    for (int l = 1; l < mg.nlev; ++l) {
        const size_t blk = (size_t)mg.lv[l].n * W * sizeof(cplx<T>);
        o_r[l] = take(blk);
        o_z[l] = take(blk);
        o_t[l] = take(blk);
        if (l < mg.nlev - 1) o_d[l] = take((size_t)mg.lv[l].n * N * sizeof(cplx<T>));
    }
    const size_t o_c = take((size_t)nc * N * sizeof(cplx<T>));
    CKS(ensure(h, h->mgState, off));
    char *base = reinterpret_cast<char *>(h->mgState.p);
    mg.lv[0].dinv = kb.dinv;
    for (int l = 1; l < mg.nlev; ++l) {
        mg.lv[l].r = reinterpret_cast<cplx<T> *>(base + o_r[l]);
        mg.lv[l].z = reinterpret_cast<cplx<T> *>(base + o_z[l]);
        mg.lv[l].t = reinterpret_cast<cplx<T> *>(base + o_t[l]);
        mg.lv[l].dinv = l < mg.nlev - 1 ? reinterpret_cast<cplx<T> *>(base + o_d[l]) : nullptr;
    }
    mg.cinv = reinterpret_cast<cplx<T> *>(base + o_c);
    mg.Minv = nullptr;
    if (e_inv >= 0) {
        if constexpr (sizeof(T) == 4) {
            if (!h->cublas) {
                if (cublasCreate(&h->cublas) != CUBLAS_STATUS_SUCCESS) {
                    h->cublas = nullptr;
                    g_last_error = "cublasCreate failed";
                    return SLRF_ECUDA;
                }
            }
            const size_t inv_bytes = (size_t)N * nc * nc * sizeof(cplx<T>);
            const size_t inv_off = (inv_bytes + 255) / 256 * 256;
            CKS(ensure(h, h->mgInv, inv_off + coarse_inverse_work_bytes(nc, N)));
            float2 *Minv = reinterpret_cast<float2 *>(h->mgInv.p);
            std::vector<double> key = {(double)e_inv, (double)nc, (double)h->mg_gen, (double)N};
            for (int j = 0; j < N; ++j) {
                key.push_back(f->sigma_re[j]);
                key.push_back(f->sigma_im[j]);
            }
            if (key != h->inv_key || h->inv_buf != h->mgInv.p) {
                const MgLevel<T> &Le = mg.lv[e_inv];
                const int rc = coarse_inverse(h->ctx, h->cublas, nc, make_poleset<float>(f), Le.gptr, Le.gcol,
                                              reinterpret_cast<const float2 *>(Le.ab), Minv,
                                              reinterpret_cast<char *>(h->mgInv.p) + inv_off);
                if (rc != 0) {
                    h->inv_key.clear();
                    g_last_error = "coarse inverse: cuBLAS status " + std::to_string(rc);
                    return SLRF_ECUDA;
                }
                h->inv_key = key;
                h->inv_buf = h->mgInv.p;
                h->inv_pan_ok = false;
            }
            mg.Minv = reinterpret_cast<const cplx<T> *>(Minv);
            mg.cublas = h->cublas;
            mg.Mpan = nullptr;
            if (h->opts.mg_exact_tc && coarse_tc_fits(d.Lp)) {
                CKS(ensure(h, h->mgInvPan, coarse_tc_panel_bytes(nc, N)));
                CKS(ensure(h, h->mgCtWork, coarse_tc_work_bytes(nc, N, d.Lp)));
                if (!h->inv_pan_ok || h->inv_pan_buf != h->mgInvPan.p) {
                    coarse_tc_panels(h->ctx, nc, N, Minv, h->mgInvPan.p);
                    h->inv_pan_ok = true;
                    h->inv_pan_buf = h->mgInvPan.p;
                }
                mg.Mpan = h->mgInvPan.p;
                mg.ct_work = h->mgCtWork.p;
                mg.ct_err = h->d_pin + 1;
            }
        }
        mg_dinv<T>(h->ctx, mg, make_poleset<T>(f));
        return SLRF_OK;
    }
    // the previous solve of this handle synchronised before returning, so the
    // staging vector is free to be rewritten
    h->mg_cinv_host.resize((size_t)nc * N * sizeof(cplx<T>));
    cplx<T> *ci = reinterpret_cast<cplx<T> *>(h->mg_cinv_host.data());
    for (int k = 0; k < nc; ++k)
        for (int j = 0; j < N; ++j) {
            const cd v = 1.0 / (cd((*lam)[k], 0.0) - cd(f->sigma_re[j], f->sigma_im[j]));
            ci[(size_t)k * N + j] = mk((T)v.real(), (T)v.imag());
        }
    CK(cudaMemcpyAsync(mg.cinv, ci, h->mg_cinv_host.size(), cudaMemcpyHostToDevice, h->ctx.stream));
    mg_dinv<T>(h->ctx, mg, make_poleset<T>(f));
    return SLRF_OK;
}

// ---------------------------------------------------------------------------
// Krylov solve of all (pole, column) systems; filter output accumulated in Uacc
// ---------------------------------------------------------------------------
struct KStats {
    int64_t iters_max = 0;        // iterations of the longest column
    int64_t spmv = 0;             // sum over columns of iterations
    double iters_per_pole[SLRF_MAX_POLES] = {};
    int n_fail = 0;               // columns that hit the cap or broke down
    int n_breakdown = 0;
    int mg_levels = 0;            // multigrid levels used (0: none)
};

// ILU preconditioner of one call: the pattern arrays once per handle (host
// build from the device CSR), the factors of this call's poles.
template <typename T>
slrf_status ilu_prepare(slrf_handle *h, const slrf_filter *f, const KrylovDims &d, IluFactor<T> &fac) {
    Ctx &ctx = h->ctx;
    const int n = h->A.n;
    if (!h->ilu_ready) {
        std::vector<int32_t> rp(n + 1), ci(h->A.nnz);
        CK(cudaMemcpyAsync(rp.data(), h->A.rowptr, (n + 1) * sizeof(int32_t), cudaMemcpyDeviceToHost, ctx.stream));
        CK(cudaMemcpyAsync(ci.data(), h->A.col, h->A.nnz * sizeof(int32_t), cudaMemcpyDeviceToHost, ctx.stream));
        CK(cudaStreamSynchronize(ctx.stream));
        int64_t nnzl = 0;
        const std::vector<int32_t> v = ilu_pattern_host(n, rp, ci, &nnzl);
        CKS(ensure(h, h->iluPat, v.size() * sizeof(int32_t)));
        CK(cudaMemcpyAsync(h->iluPat.p, v.data(), v.size() * sizeof(int32_t), cudaMemcpyHostToDevice, ctx.stream));
        CK(cudaStreamSynchronize(ctx.stream));   // pageable source
        ilu_pattern_views(as<int32_t>(h->iluPat), n, nnzl, h->ilu_pat);
        h->ilu_ready = true;
    }
    const int N = f->n_poles;
    const size_t work = (ilu_factor_work_bytes(h->ilu_pat, N) + 255) / 256 * 256;
    const size_t outb = ((size_t)N * h->ilu_pat.nnzl + (size_t)n * N) * sizeof(cplx<T>);
    CKS(ensure(h, h->iluFac, work + outb));
    CKS(ensure(h, h->kIluY, (size_t)n * d.W() * sizeof(cplx<T>)));
    ilu_factor<T>(ctx, h->A, h->ilu_pat, make_poleset<double>(f), h->opts.ilu_sweeps, h->iluFac.p,
                  reinterpret_cast<cplx<T> *>(reinterpret_cast<char *>(h->iluFac.p) + work), fac);
    return SLRF_OK;
}

// SELL-C-sigma form of the handle's pencil (shape from the options); no-op
// if built.  An allocation failure leaves the handle without the form (the
// row-group kernel runs instead).
slrf_status sell_upload(slrf_handle *h, const std::vector<int32_t> &rp, const std::vector<int32_t> &ci,
                        const std::vector<double> &av, const std::vector<double> &bv) {
    DevPencil &A = h->A;
    if (A.sell_ab) return SLRF_OK;
    const int C = h->opts.sell_c ? h->opts.sell_c : 32, sg = h->opts.sell_sigma ? h->opts.sell_sigma : 256;
    std::vector<int32_t> cptr, scol, perm, rlen;
    std::vector<float2> sab;
    if (!build_sell(A.n, rp, ci, av, bv, C, sg, cptr, scol, sab, perm, rlen)) return SLRF_OK;
    cudaStream_t s = h->ctx.stream;
    void **bufs[] = {(void **)&A.sell_cptr, (void **)&A.sell_col, (void **)&A.sell_ab, (void **)&A.sell_perm,
                     (void **)&A.sell_rlen};
    const size_t bytes[] = {cptr.size() * 4, scol.size() * 4, sab.size() * 8, perm.size() * 4, rlen.size() * 4};
    const void *src[] = {cptr.data(), scol.data(), sab.data(), perm.data(), rlen.data()};
    for (int i = 0; i < 5; ++i) {
        if (dev_alloc(h, bufs[i], bytes[i]) != cudaSuccess) {
            cudaGetLastError();
            *bufs[i] = nullptr;
            for (int k = 0; k < i; ++k) {
                cudaFreeAsync(*bufs[k], s);
                *bufs[k] = nullptr;
            }
            return SLRF_OK;
        }
        h->pencil_bytes += bytes[i];
    }
    for (int i = 0; i < 5; ++i) CK(cudaMemcpyAsync(*bufs[i], src[i], bytes[i], cudaMemcpyHostToDevice, s));
    A.sell_c = C;
    A.sell_sigma = sg;
    A.sell_nchunks = (int)(cptr.size() - 1);
    A.sell_slots = cptr.back();
    CK(cudaStreamSynchronize(s));   // pageable sources
    return SLRF_OK;
}

// the same from the device copy of the pencil
slrf_status ensure_sell(slrf_handle *h) {
    if (h->A.sell_ab) return SLRF_OK;
    const int64_t n = h->A.n, nnz = h->A.nnz;
    std::vector<int32_t> rp(n + 1), ci(nnz);
    std::vector<double> av(nnz), bv(nnz);
    cudaStream_t s = h->ctx.stream;
    CK(cudaMemcpyAsync(rp.data(), h->A.rowptr, (n + 1) * 4, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(ci.data(), h->A.col, nnz * 4, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(av.data(), h->A.a, nnz * 8, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(bv.data(), h->A.b, nnz * 8, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return sell_upload(h, rp, ci, av, bv);
}

// Kernel choice of the FP32 shifted product (slrf_opts.spmm_kernel = 0):
// the candidate kernels are timed on this solve's blocks (one warm launch,
// then three timed ones each) and the fastest is kept, per device, pattern
// and column count, for the rest of the process.
std::mutex g_tune_mu;
std::map<std::array<int64_t, 7>, int> g_tune;

template <typename T>
slrf_status resolve_spmm_kernel(slrf_handle *h, const KrylovDims &d, KrylovBuffers<T> &kb, const cplx<T> *sig) {
    DevPencil &A = h->A;
    if (sizeof(T) != 4) return SLRF_OK;
    if (A.spmm_kind == SPMM_SELL) CKS(ensure_sell(h));
    // a requested form the pencil does not have runs as the row-group kernel
    if ((A.spmm_kind == SPMM_STAGED && spmm_staged_smem(A) == 0) || (A.spmm_kind == SPMM_NODEBLOCK && !A.nb_coef) ||
        (A.spmm_kind == SPMM_SELL && !A.sell_ab))
        A.spmm_kind = SPMM_ROWGROUP;
    if (A.spmm_kind != 0) return SLRF_OK;
    const int sell_c = h->opts.sell_c ? h->opts.sell_c : 32, sell_sigma = h->opts.sell_sigma ? h->opts.sell_sigma : 256;
    const std::array<int64_t, 7> key = {h->device, A.n, A.nnz, A.rg_rows, A.rg_nnz, d.W(),
                                        (int64_t)sell_c * 1000000 + sell_sigma};
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto it = g_tune.find(key);
        if (it != g_tune.end()) {
            A.spmm_kind = it->second;
            if (A.spmm_kind == SPMM_SELL) CKS(ensure_sell(h));
            if (A.spmm_kind == SPMM_SELL && !A.sell_ab) A.spmm_kind = SPMM_ROWGROUP;
            return SLRF_OK;
        }
    }
    // first timing for this pattern: every form is a candidate; node pencils
    // time row groups against node blocks (the staged kernel, bulk-copying
    // 81-entry union lists, measured ~10x slower than either)
    CKS(ensure_sell(h));
    std::vector<int> kinds = {SPMM_ROWGROUP};
    if (A.nb_coef) kinds.push_back(SPMM_NODEBLOCK);
    else if (spmm_staged_smem(A) > 0) kinds.push_back(SPMM_STAGED);
    if (A.sell_ab) kinds.push_back(SPMM_SELL);
    if (kinds.size() == 1) {
        A.spmm_kind = SPMM_ROWGROUP;
        return SLRF_OK;
    }
    Ctx &ctx = h->ctx;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        g_last_error = "autotune: event creation failed";
        return SLRF_ECUDA;
    }
    float best = 0.f;
    int pick = SPMM_ROWGROUP;
    for (int kind : kinds) {
        A.spmm_kind = kind;
        krylov_spmm<T>(ctx, d, A, sig, kb.P, kb.Q, kb.s.flag, kb.s.part, kb.gy);
        cudaEventRecord(e0, ctx.stream);
        for (int r = 0; r < 3; ++r) krylov_spmm<T>(ctx, d, A, sig, kb.P, kb.Q, kb.s.flag, kb.s.part, kb.gy);
        cudaEventRecord(e1, ctx.stream);
        float ms = 0.f;
        const cudaError_t err = cudaEventSynchronize(e1);
        if (err == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
        if (err != cudaSuccess || *(volatile int32_t *)(h->h_pin + 1) != 0) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            g_last_error = err != cudaSuccess ? std::string("autotune: ") + cudaGetErrorString(err)
                                              : std::string("autotune: a bounded device wait gave up");
            return err != cudaSuccess ? SLRF_ECUDA : SLRF_ETIMEOUT;
        }
        if (kind == SPMM_ROWGROUP || ms < best) {
            best = ms;
            pick = kind;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    A.spmm_kind = pick;
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune[key] = pick;
    return SLRF_OK;
}

template <typename T>
slrf_status krylov_solve(slrf_handle *h, const slrf_filter *f, int m, const double *rhs, int64_t ldr,
                         const std::vector<int> &col_active, const std::vector<cd> &coef, double tol, int maxit,
                         KrylovBuffers<T> &kb, KrylovDims &d, KStats &st) {
    Ctx &ctx = h->ctx;
    const int N = f->n_poles;
    d.n = h->A.n;
    d.N = N;
    d.m = m;
    d.Lp = (m + 1) / 2 * 2;
    const int W = d.W();
    const int64_t n = d.n;
    kb.gy = krylov_row_groups(ctx, d, sizeof(T) == 4);
    *(volatile int32_t *)(h->h_pin + 1) = 0;   // device-side wait timeouts of this solve
    CKS(ensure(h, h->kP, (size_t)n * W * sizeof(cplx<T>)));
    CKS(ensure(h, h->kQ, (size_t)n * W * sizeof(cplx<T>)));
    CKS(ensure(h, h->kR, (size_t)n * W * sizeof(cplx<T>)));
    CKS(ensure(h, h->kDinv, (size_t)n * N * sizeof(cplx<T>)));
    CKS(ensure(h, h->kU, (size_t)n * d.Lp * sizeof(T)));
    CKS(ensure(h, h->kPart, (size_t)kb.gy * W * 4 * sizeof(T)));
    CKS(ensure(h, h->kSig, SLRF_MAX_POLES * sizeof(cplx<T>)));
    // scalars: alpha, rho, beta, ua (cplx<T>) ; bnorm2, rnorm2 (double) ; coef (double2) ; flag, iters (int)
    const size_t sc_bytes = (size_t)W * (4 * sizeof(cplx<T>) + 2 * sizeof(double) + sizeof(double2)) + 64;
    CKS(ensure(h, h->kScal, sc_bytes));
    CKS(ensure(h, h->kFlags, (size_t)W * 2 * sizeof(int32_t) + 64));

    kb.P = as<cplx<T>>(h->kP);
    kb.Q = as<cplx<T>>(h->kQ);
    kb.R = as<cplx<T>>(h->kR);
    kb.dinv = as<cplx<T>>(h->kDinv);
    kb.Uacc = as<T>(h->kU);
    kb.s.part = as<T>(h->kPart);
    char *p = reinterpret_cast<char *>(h->kScal.p);
    kb.s.alpha = reinterpret_cast<cplx<T> *>(p);
    p += (size_t)W * sizeof(cplx<T>);
    kb.s.rho = reinterpret_cast<cplx<T> *>(p);
    p += (size_t)W * sizeof(cplx<T>);
    kb.s.beta = reinterpret_cast<cplx<T> *>(p);
    p += (size_t)W * sizeof(cplx<T>);
    kb.s.ua = reinterpret_cast<cplx<T> *>(p);
    p += (size_t)W * sizeof(cplx<T>);
    kb.s.bnorm2 = reinterpret_cast<double *>(p);
    p += (size_t)W * sizeof(double);
    kb.s.rnorm2 = reinterpret_cast<double *>(p);
    p += (size_t)W * sizeof(double);
    kb.s.coef = reinterpret_cast<double2 *>(p);
    kb.s.flag = as<int32_t>(h->kFlags);
    kb.s.iters = kb.s.flag + W;
    kb.s.active_count = nullptr;

    // host-side per-column setup
    std::vector<int32_t> flags(W, 0);
    std::vector<double2> cf(W);
    for (int j = 0; j < N; ++j)
        for (int c = 0; c < d.Lp; ++c) {
            const int col = j * d.Lp + c;
            flags[col] = (c < m) ? (col_active[c] ? 1 : 4) : 0;
            const cd v = (c < m) ? coef[(size_t)j * m + c] : cd(0, 0);
            cf[col] = make_double2(v.real(), v.imag());
        }
    CK(cudaMemcpyAsync(kb.s.flag, flags.data(), W * sizeof(int32_t), cudaMemcpyHostToDevice, ctx.stream));
    CK(cudaMemcpyAsync(kb.s.coef, cf.data(), W * sizeof(double2), cudaMemcpyHostToDevice, ctx.stream));
    std::vector<cplx<T>> sg(SLRF_MAX_POLES);
    for (int j = 0; j < N; ++j) sg[j] = mk((T)f->sigma_re[j], (T)f->sigma_im[j]);
    CK(cudaMemcpyAsync(h->kSig.p, sg.data(), N * sizeof(cplx<T>), cudaMemcpyHostToDevice, ctx.stream));
    // the host vectors above are pageable; make the copies complete before they go out of scope
    bool use_mg = uses_mg(h);
    const bool bcg = h->opts.krylov == SLRF_KRYLOV_BICGSTAB;
    kb.Z = nullptr;
    BcgBuffers<T> bb{};
    if (bcg) {
        const size_t blk = (size_t)n * W * sizeof(cplx<T>);
        CKS(ensure(h, h->kBcg, 5 * blk + 2 * (size_t)W * sizeof(cplx<T>)));
        char *q = reinterpret_cast<char *>(h->kBcg.p);
        bb.Rh = reinterpret_cast<cplx<T> *>(q);
        bb.V = reinterpret_cast<cplx<T> *>(q + blk);
        bb.Y = reinterpret_cast<cplx<T> *>(q + 2 * blk);
        bb.Z = reinterpret_cast<cplx<T> *>(q + 3 * blk);
        bb.Tt = reinterpret_cast<cplx<T> *>(q + 4 * blk);
        bb.omega = reinterpret_cast<cplx<T> *>(q + 5 * blk);
        bb.ua2 = bb.omega + W;
    }
    if (use_mg) {
        bool usable = true;
        CKS(mg_prepare<T>(h, f, d, kb, h->opts.precond == SLRF_PRECOND_AUTO, &usable));
        use_mg = usable;
    }
    const bool use_ilu = !use_mg && h->opts.precond == SLRF_PRECOND_ILU;
    IluFactor<T> ilu{};
    if (use_ilu) CKS(ilu_prepare<T>(h, f, d, ilu));
    cplx<T> *ilu_y = use_ilu ? as<cplx<T>>(h->kIluY) : nullptr;
    if ((use_mg || use_ilu) && !bcg) {
        CKS(ensure(h, h->kZ, (size_t)n * W * sizeof(cplx<T>)));
        kb.Z = as<cplx<T>>(h->kZ);
    }
    if (use_mg) {
        // the update forms the cycle's gathered block y = D r (finest level)
        if (!bcg && mg_of<T>(h).nlev > 1) kb.mgd = mg_of<T>(h).lv[0].dinv;
    } else {
        const PoleSet<T> ps = make_poleset<T>(f);
        krylov_dinv<T>(ctx, h->A, ps, h->opts.precond == SLRF_PRECOND_NONE ? SLRF_PRECOND_NONE : SLRF_PRECOND_JACOBI,
                       kb.dinv);
    }
    const cplx<T> *sig = as<cplx<T>>(h->kSig);
    fill_zero(ctx, kb.Uacc, (size_t)n * d.Lp * sizeof(T));
    krylov_init<T>(ctx, d, kb, rhs, ldr, nullptr);
    if (bcg) {
        bicgstab_init<T>(ctx, d, kb, bb);
    } else if (use_mg) {
        mg_apply<T>(ctx, d, mg_of<T>(h), sig, kb.s.flag, kb.s.part, kb.gy, kb.R, kb.Z, kb.Q);
        krylov_direction<T>(ctx, d, kb, 1);
    } else if (use_ilu) {
        ilu_apply<T>(ctx, d, h->ilu_pat, ilu, h->opts.ilu_tri_sweeps, kb.gy, kb.s.flag, kb.R, kb.Z, kb.Q, ilu_y,
                     kb.s.part);
        krylov_direction<T>(ctx, d, kb, 1);
    }
    krylov_reduce_init<T>(ctx, d, kb);
    CKS(resolve_spmm_kernel<T>(h, d, kb, sig));

    int n_active = 0;
    for (int col = 0; col < W; ++col) n_active += flags[col] == 1;
    d.frac = (double)n_active / W;
    const double tol2 = tol * tol;
    const int every = std::max(1, h->opts.check_every);
    int it = 0;
    for (; it < maxit;) {
        const int chunk = std::min(every, maxit - it);
        for (int k = 0; k < chunk && bcg; ++k) {
            // y = M^{-1} p ; v = A y ; alpha ; s = r - alpha v ; z = M^{-1} s ; t = A z ; omega ;
            // x, r ; rho', beta ; p
            if (use_mg)
                mg_apply<T>(ctx, d, mg_of<T>(h), sig, kb.s.flag, kb.s.part, kb.gy, kb.P, bb.Y, bb.Tt);
            else if (use_ilu)
                ilu_apply<T>(ctx, d, h->ilu_pat, ilu, h->opts.ilu_tri_sweeps, kb.gy, kb.s.flag, kb.P, bb.Y, bb.Tt,
                             ilu_y, nullptr);
            else
                bicgstab_precond_jacobi<T>(ctx, d, kb, kb.P, bb.Y);
            krylov_spmm<T>(ctx, d, h->A, sig, bb.Y, bb.V, kb.s.flag, kb.s.part, kb.gy);
            bicgstab_alpha<T>(ctx, d, kb, bb);
            bicgstab_s<T>(ctx, d, kb, bb, !use_mg && !use_ilu);
            if (use_mg) mg_apply<T>(ctx, d, mg_of<T>(h), sig, kb.s.flag, kb.s.part, kb.gy, kb.R, bb.Z, bb.Tt);
            if (use_ilu)
                ilu_apply<T>(ctx, d, h->ilu_pat, ilu, h->opts.ilu_tri_sweeps, kb.gy, kb.s.flag, kb.R, bb.Z, bb.Tt,
                             ilu_y, nullptr);
            krylov_spmm<T>(ctx, d, h->A, sig, bb.Z, bb.Tt, kb.s.flag, kb.s.part, kb.gy);
            bicgstab_omega<T>(ctx, d, kb, bb);
            bicgstab_update<T>(ctx, d, kb, bb);
            krylov_reduce_beta<T>(ctx, d, kb, tol2, maxit);
            bicgstab_direction<T>(ctx, d, kb, bb);
        }
        for (int k = 0; k < chunk && !bcg; ++k) {
            krylov_spmm<T>(ctx, d, h->A, sig, kb.P, kb.Q, kb.s.flag, kb.s.part, kb.gy);
            krylov_reduce_alpha<T>(ctx, d, kb);
            krylov_update<T>(ctx, d, kb);
            if (use_mg) mg_apply<T>(ctx, d, mg_of<T>(h), sig, kb.s.flag, kb.s.part, kb.gy, kb.R, kb.Z, kb.Q, kb.Q);
            if (use_ilu)
                ilu_apply<T>(ctx, d, h->ilu_pat, ilu, h->opts.ilu_tri_sweeps, kb.gy, kb.s.flag, kb.R, kb.Z, kb.Q,
                             ilu_y, kb.s.part);
            krylov_reduce_beta<T>(ctx, d, kb, tol2, maxit);
            krylov_direction<T>(ctx, d, kb);
        }
        it += chunk;
        krylov_count_active(ctx, W, kb.s.flag, h->d_pin);   // mapped pinned host word
        CK(cudaEventRecord(h->ev_poll, ctx.stream));
        CK(cudaEventSynchronize(h->ev_poll));
        n_active = *(volatile int32_t *)h->h_pin;
        if (*(volatile int32_t *)(h->h_pin + 1) != 0) {
            g_last_error = "shifted product: a bounded device wait gave up";
            return SLRF_ETIMEOUT;
        }
        d.frac = (double)n_active / W;
        if (n_active == 0) break;
    }
    CK(cudaGetLastError());
    // statistics
    std::vector<int32_t> fl(W), its(W);
    CK(cudaMemcpyAsync(fl.data(), kb.s.flag, W * sizeof(int32_t), cudaMemcpyDeviceToHost, ctx.stream));
    CK(cudaMemcpyAsync(its.data(), kb.s.iters, W * sizeof(int32_t), cudaMemcpyDeviceToHost, ctx.stream));
    CK(cudaStreamSynchronize(ctx.stream));
    st = KStats();
    st.mg_levels = use_mg ? mg_of<T>(h).nlev : 0;
    for (int j = 0; j < N; ++j) {
        int64_t s = 0, cnt = 0;
        for (int c = 0; c < m; ++c) {
            const int col = j * d.Lp + c;
            s += its[col];
            st.iters_max = std::max<int64_t>(st.iters_max, its[col]);
            if (fl[col] == 4) continue;
            ++cnt;
            if (fl[col] == 1 || fl[col] == 3) ++st.n_fail;
            if (fl[col] == 2) ++st.n_breakdown;
        }
        st.spmv += bcg ? 2 * s : s;
        st.iters_per_pole[j] = cnt ? (double)s / cnt : 0.0;
    }
    return SLRF_OK;
}

// G = X^T Y with the handle's Gram method (Ozaki digits on the tcgen05 or the
// mma.sync tensor path, or FP64) (symmetric: Y = B X with B symmetric, so only
// the upper tiles are computed)
slrf_status gram(slrf_handle *h, int64_t n, int m, const double *X, int64_t ldx, const double *Y, int64_t ldy,
                 double *G, bool symmetric = false) {
    Ctx &ctx = h->ctx;
    if (h->opts.gram_ozaki) {
        CKS(ensure(h, h->rOz, ozaki_gram_work_bytes(n, m, ctx.sm_count)));
        ozaki_gram(ctx, n, m, X, ldx, Y, ldy, G, h->rOz.p, symmetric,
                   h->opts.gram_ozaki == 2 ? h->d_pin + 1 : nullptr);
        return SLRF_OK;
    }
    const int split = gram_split(ctx, m, n);
    CKS(ensure(h, h->rSplit, (size_t)split * m * m * sizeof(double)));
    dgemm(ctx, 1, 0, m, m, (int)n, X, ldx, Y, ldy, 0.0, G, m, split, as<double>(h->rSplit), KC_GRAM);
    return SLRF_OK;
}

// C = (A diag(cs)) B for a tall A (n x k) and a small B (k x m): FP64-accurate
// int8 tensor-core digits with the handle's Ozaki option, else the FP64 tile
// GEMM (cs applied to the rows of B in place; B is scratch of the caller).
slrf_status tall_product(slrf_handle *h, int64_t n, int k, int m, const double *A, int64_t lda, const double *cs,
                         double *B, int64_t ldb, double *C, int64_t ldc) {
    Ctx &ctx = h->ctx;
    if (h->opts.gram_ozaki && ozaki_tall_fits(k)) {
        CKS(ensure(h, h->rOzT, ozaki_tall_work_bytes(n, k, m)));
        ozaki_tall(ctx, n, k, m, A, lda, cs, B, ldb, C, ldc, h->rOzT.p, KC_TALL_GEMM,
                   h->opts.gram_ozaki == 2 ? h->d_pin + 1 : nullptr);
        return SLRF_OK;
    }
    if (cs) small_scale_rows(ctx, k, cs, B);
    dgemm(ctx, 0, 0, (int)n, m, k, A, lda, B, ldb, 0.0, C, ldc, 1, nullptr, KC_TALL_GEMM);
    return SLRF_OK;
}

// ---------------------------------------------------------------------------
// Cholesky-QR2 + Rayleigh-Ritz of span(U): theta (ascending), X = U M, AX, BX
// (all n x m with leading dimension m except U/X which take ldu/ldx)
// ---------------------------------------------------------------------------
slrf_status rr_step(slrf_handle *h, int m, const double *U, int64_t ldu, double *theta, double *X, int64_t ldx,
                    double *AX, double *BX, int32_t *chol_status) {
    Ctx &ctx = h->ctx;
    *(volatile int32_t *)(h->h_pin + 1) = 0;   // device-side wait timeouts of this step
    *(volatile int32_t *)(h->h_pin + 2) = 0;   // pass 1's Cholesky status
    const int64_t n = h->A.n;
    const size_t m2 = (size_t)m * m;
    const int split = gram_split(ctx, m, n);
    CKS(ensure(h, h->rW1, (size_t)n * m * sizeof(double)));
    CKS(ensure(h, h->rQ1, (size_t)n * m * sizeof(double)));
    CKS(ensure(h, h->rSplit, (size_t)split * m2 * sizeof(double)));
    CKS(ensure(h, h->rSmall, (8 * m2 + 4 * (size_t)m) * sizeof(double) + small_syev_work_bytes(m) + 64));
    double *W1 = as<double>(h->rW1), *Q1 = as<double>(h->rQ1), *spw = as<double>(h->rSplit);
    double *G = as<double>(h->rSmall);
    double *R1 = G + m2, *T1 = R1 + m2, *T2 = T1 + m2, *Ah = T2 + m2, *Ah1 = Ah + m2, *Sm = Ah1 + m2,
           *Mm = Sm + m2, *s = Mm + m2;
    int32_t *st = reinterpret_cast<int32_t *>(s + 2 * m);
    double *syw = reinterpret_cast<double *>(reinterpret_cast<char *>(s + 4 * m));

    // pass 1: G = U^T B U, column scaling, R1 = chol, T1 = S R1^{-1}, Q1 = U T1.
    // If the scaled Gram is not numerically positive definite, R1 comes from
    // G + s I with the shifted Cholesky-QR shift s = 11 (n m + m (m + 1)) u
    // ||U S||^2 (Fukaya et al., SIAM J. Sci. Comput. 2020; ||U S||^2 <= m after
    // the column scaling) and a third pass follows (shifted Cholesky-QR3).
    const double shift = 11.0 * ((double)n * m + (double)m * (m + 1)) * 1.1102230246251565e-16 * m;
    // mapped (third word of the handle's poll slot; the second one collects
    // the bounded-wait timeouts of the tensor-core kernels): the host reads
    // it after pass 1
    int32_t *pin_status = h->d_pin + 2;
    spmm_real(ctx, h->A, m, U, ldu, nullptr, 0, W1, m);
    CKS(gram(h, n, m, U, ldu, W1, m, G, true));
    small_colscale(ctx, m, G, s);
    small_chol_upper(ctx, m, G, R1, pin_status, shift);
    small_triinv_upper(ctx, m, R1, T1);
    // Q1 = (U S) R1^{-1}: the column scaling S makes the split operand well scaled
    CKS(tall_product(h, n, m, m, U, ldu, s, T1, m, Q1, m));
    CK(cudaEventRecord(h->ev_poll, ctx.stream));
    CK(cudaEventSynchronize(h->ev_poll));
    if (*(volatile int32_t *)(h->h_pin + 1) != 0) {
        g_last_error = "projection step: a bounded device wait gave up";
        return SLRF_ETIMEOUT;
    }
    const int32_t st1 = *(volatile int32_t *)(h->h_pin + 2);
    if (st1 > 0) {
        if (chol_status) {
            chol_status[0] = st1;
            chol_status[1] = 0;
        }
        return SLRF_OK;   // reported as SLRF_CHOLQR_FAIL by the caller
    }
    if (st1 < 0) {
        // extra pass on the shifted factor: Q1 <- Q1 R^{-1} with R = chol(Q1^T B Q1)
        CKS(ensure(h, h->rQ2, (size_t)n * m * sizeof(double)));
        double *Q2 = as<double>(h->rQ2);
        spmm_real(ctx, h->A, m, Q1, m, nullptr, 0, W1, m);
        CKS(gram(h, n, m, Q1, m, W1, m, G, true));
        small_chol_upper(ctx, m, G, G, st + 2, 0.0);
        small_triinv_upper(ctx, m, G, T1);
        CKS(tall_product(h, n, m, m, Q1, m, nullptr, T1, m, Q2, m));
        CK(cudaMemcpyAsync(Q1, Q2, (size_t)n * m * sizeof(double), cudaMemcpyDeviceToDevice, ctx.stream));
        h->shifted_cholqr += 1;
    } else {
        CK(cudaMemsetAsync(st + 2, 0, sizeof(int32_t), ctx.stream));
    }
    // pass 2: G2 = Q1^T B Q1, R2 = chol, T2 = R2^{-1}
    spmm_real(ctx, h->A, m, Q1, m, nullptr, 0, W1, m);
    CKS(gram(h, n, m, Q1, m, W1, m, G, true));
    small_chol_upper(ctx, m, G, G, st + 1, 0.0);
    small_triinv_upper(ctx, m, G, T2);
    // projected A: A_hat = T2^T (Q1^T A Q1) T2
    spmm_real(ctx, h->A, m, Q1, m, W1, m, nullptr, 0);
    CKS(gram(h, n, m, Q1, m, W1, m, Ah1, true));
    dgemm(ctx, 0, 0, m, m, m, Ah1, m, T2, m, 0.0, R1, m, 1, nullptr, KC_SMALL_DENSE);
    dgemm(ctx, 1, 0, m, m, m, T2, m, R1, m, 0.0, Ah, m, 1, nullptr, KC_SMALL_DENSE);
    ctx.before(KC_SMALL_DENSE, 16.0 * m2, 0);
    k_symmetrize<<<(unsigned)((m2 + 255) / 256), 256, 0, ctx.stream>>>(m, Ah);
    ctx.after();
    CK(small_syev(ctx, m, Ah, theta, Sm, syw, h->opts.eig_refine));
    // X = Q1 (T2 S); AX, BX by SpMM
    dgemm(ctx, 0, 0, m, m, m, T2, m, Sm, m, 0.0, Mm, m, 1, nullptr, KC_SMALL_DENSE);
    CKS(tall_product(h, n, m, m, Q1, m, nullptr, Mm, m, X, ldx));
    spmm_real(ctx, h->A, m, X, ldx, AX, m, BX, m);
    if (chol_status) {
        // pass 2 (and the extra pass) must succeed; pass 1's status was read above
        CK(cudaMemcpyAsync(chol_status, st + 1, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, ctx.stream));
        CK(cudaStreamSynchronize(ctx.stream));
        chol_status[0] = chol_status[0] > 0 ? chol_status[0] : (chol_status[1] > 0 ? chol_status[1] : 0);
        chol_status[1] = 0;
        if (*(volatile int32_t *)(h->h_pin + 1) != 0) {
            g_last_error = "Gram: a bounded device wait gave up";
            return SLRF_ETIMEOUT;
        }
    }
    return SLRF_OK;
}

slrf_status check_dense(const void *p, int64_t ld, int32_t m) { return (p && m >= 1 && ld >= m) ? SLRF_OK : SLRF_EINVAL; }

// Algorithm 1 driver (device buffers)
slrf_status subspace_core(slrf_handle *h, const slrf_filter *f, double gamma, int L, const double *V0, int64_t ldv,
                          double tol, int max_outer, double *theta, double *X, int64_t ldx, double *resid,
                          int32_t *n_conv, slrf_report *rep) {
    Ctx &ctx = h->ctx;
    const int64_t n = h->A.n;
    const int N = f->n_poles;
    const bool mixed = h->opts.precision == SLRF_PREC_MIXED;
    CKS(ensure(h, h->rAX, (size_t)n * L * sizeof(double)));
    CKS(ensure(h, h->rBX, (size_t)n * L * sizeof(double)));
    CKS(ensure(h, h->rRes, (size_t)n * L * sizeof(double)));
    CKS(ensure(h, h->rV, (size_t)n * L * sizeof(double)));
    CKS(ensure(h, h->rRho, (size_t)L * sizeof(double) * 2 + (size_t)ctx.sm_count * 4 * L * 3 * sizeof(double) +
                               (size_t)(n + 7) / 8 * 0));
    double *AX = as<double>(h->rAX), *BX = as<double>(h->rBX), *Rm = as<double>(h->rRes), *U = as<double>(h->rV);
    double *rho_ax = as<double>(h->rRho);
    double *rwork = rho_ax + L;

    std::vector<double> th(L), rh(L), rha(L);
    std::vector<cd> coef((size_t)N * L);
    std::vector<int> active(L, 1);
    int32_t chol[2] = {0, 0};
    KStats st;
    int64_t spmv = 0, kit = 0;
    double ipp[SLRF_MAX_POLES] = {};
    int outer = 0;
    slrf_status status = SLRF_NOT_CONVERGED;
    int nw = 0, nc = 0;
    double worst = 0, worst_ax = 0, worst_all = 0;
    // stagnation: outer steps since the largest wanted residual (all Ritz pairs
    // while none is wanted yet) last fell below 0.9 of its best value
    double best_worst = HUGE_VAL;
    int since_best = 0;
    bool k64 = false;   // MIXED: Krylov solves escalated to FP64
    auto stagnated = [&]() {
        if (h->opts.stagnation_window <= 0) return false;
        const double w = nw > 0 ? worst : worst_all;
        if (w < 0.9 * best_worst) {
            best_worst = w;
            since_best = 0;
            return false;
        }
        return ++since_best >= h->opts.stagnation_window;
    };

    auto evaluate = [&]() -> slrf_status {
        residual(ctx, (int)n, L, AX, BX, L, theta, mixed ? Rm : nullptr, L, resid, rho_ax, rwork);
        CK(cudaMemcpyAsync(th.data(), theta, L * sizeof(double), cudaMemcpyDeviceToHost, ctx.stream));
        CK(cudaMemcpyAsync(rh.data(), resid, L * sizeof(double), cudaMemcpyDeviceToHost, ctx.stream));
        CK(cudaMemcpyAsync(rha.data(), rho_ax, L * sizeof(double), cudaMemcpyDeviceToHost, ctx.stream));
        CK(cudaStreamSynchronize(ctx.stream));
        CK(cudaGetLastError());
        nw = nc = 0;
        worst = worst_ax = worst_all = 0;
        for (int i = 0; i < L; ++i) {
            worst_all = std::max(worst_all, rh[i]);
            if (th[i] > 0 && th[i] <= gamma) {
                ++nw;
                if (rh[i] <= tol && rha[i] <= tol) ++nc;
                worst = std::max(worst, rh[i]);
                worst_ax = std::max(worst_ax, rha[i]);
            }
        }
        return SLRF_OK;
    };

    if (mixed) {
        // Rayleigh-Ritz on the start block gives (X, Theta) for the corrected form
        phase_begin(h, h->phase_r, h->phase_r_used);
        CKS(rr_step(h, L, V0, ldv, theta, X, ldx, AX, BX, chol));
        phase_end(h, h->phase_r, h->phase_r_used);
        CKS(evaluate());
        if (chol[0] || chol[1]) status = SLRF_CHOLQR_FAIL;
    }
    const double *V = V0;
    int64_t ldV = ldv;
    while (status != SLRF_CHOLQR_FAIL) {
        if (mixed) {
            if (nw == L) {
                status = SLRF_SUBSPACE_TOO_SMALL;
                break;
            }
            if (nw > 0 && nc == nw) {
                status = SLRF_OK;
                break;
            }
        }
        if (outer >= max_outer) {
            status = SLRF_NOT_CONVERGED;
            break;
        }
        ++outer;
        KrylovDims d;
        phase_begin(h, h->phase_k, h->phase_k_used);
        if (mixed) {
            // U = X Phi(Theta) + sum_j 2 Re(w_j (A - sigma_j B)^{-1} R D_j)
            std::vector<double> phi(L, 0.0);
            for (int c = 0; c < L; ++c) {
                active[c] = rh[c] > h->opts.lock_tol ? 1 : 0;
                for (int j = 0; j < N; ++j) {
                    const cd w(f->w_re[j], f->w_im[j]), sg(f->sigma_re[j], f->sigma_im[j]);
                    const cd dj = 1.0 / (th[c] - sg);
                    coef[(size_t)j * L + c] = w * dj;
                    phi[c] += 2.0 * (w * dj).real();
                }
            }
            CKS(ensure(h, h->rTheta, (size_t)L * sizeof(double)));
            CK(cudaMemcpyAsync(h->rTheta.p, phi.data(), L * sizeof(double), cudaMemcpyHostToDevice, ctx.stream));
            if (!k64) {
                KrylovBuffers<float> kb;
                CKS(krylov_solve<float>(h, f, L, Rm, L, active, coef, h->opts.inner_tol, h->opts.inner_maxit, kb, d,
                                        st));
                filter_combine<float>(ctx, (int)n, L, X, ldx, as<double>(h->rTheta), kb.Uacc, d.Lp, U, L);
            } else {
                KrylovBuffers<double> kb;
                CKS(krylov_solve<double>(h, f, L, Rm, L, active, coef, h->opts.inner_tol, h->opts.inner_maxit, kb, d,
                                         st));
                filter_combine<double>(ctx, (int)n, L, X, ldx, as<double>(h->rTheta), kb.Uacc, d.Lp, U, L);
            }
            CK(cudaStreamSynchronize(ctx.stream));   // phi is pageable host memory
        } else {
            // F = B V ; U = sum_j 2 Re(w_j (A - sigma_j B)^{-1} F)
            if (outer == 1) spmm_real(ctx, h->A, L, V, ldV, nullptr, 0, BX, L);
            for (int j = 0; j < N; ++j)
                for (int c = 0; c < L; ++c) coef[(size_t)j * L + c] = cd(f->w_re[j], f->w_im[j]);
            KrylovBuffers<double> kb;
            CKS(krylov_solve<double>(h, f, L, BX, L, active, coef, h->opts.inner_tol, h->opts.inner_maxit, kb, d,
                                     st));
            filter_combine<double>(ctx, (int)n, L, nullptr, 0, nullptr, kb.Uacc, d.Lp, U, L);
        }
        phase_end(h, h->phase_k, h->phase_k_used);
        spmv += st.spmv;
        kit += st.iters_max;
        for (int j = 0; j < N; ++j) ipp[j] += st.iters_per_pole[j];
        phase_begin(h, h->phase_r, h->phase_r_used);
        CKS(rr_step(h, L, U, L, theta, X, ldx, AX, BX, chol));
        phase_end(h, h->phase_r, h->phase_r_used);
        CKS(evaluate());
        if (chol[0] || chol[1]) {
            status = SLRF_CHOLQR_FAIL;
            break;
        }
        if (!(nw > 0 && nc == nw) && stagnated()) {
            // The FP32 corrections of the mixed form contract only while
            // kappa(A - sigma B) eps_32 < 1; past that the iteration stalls.
            // Continue with FP64 Krylov solves of the same corrected form
            // before giving up.
            if (mixed && !k64) {
                k64 = true;
                best_worst = HUGE_VAL;
                since_best = 0;
            } else {
                status = SLRF_STAGNATION;
                break;
            }
        }
        if (!mixed) {
            if (nw == L) {
                status = SLRF_SUBSPACE_TOO_SMALL;
                break;
            }
            if (nw > 0 && nc == nw) {
                status = SLRF_OK;
                break;
            }
            V = X;
            ldV = ldx;
        }
    }
    if (n_conv) *n_conv = nc;
    if (rep) {
        rep->outer_iters = outer;
        rep->n_wanted = nw;
        rep->n_conv = nc;
        rep->max_resid = worst;
        rep->max_resid_ax = worst_ax;
        rep->krylov_iters = kit;
        rep->spmv = spmv;
        rep->mg_levels = st.mg_levels;
        rep->krylov_fp64 = k64 ? 1 : 0;
        rep->spmm_kernel = h->A.spmm_kind;
        for (int j = 0; j < N; ++j) rep->iters_per_pole[j] = outer ? ipp[j] / outer : 0.0;
    }
    return status;
}

}  // namespace

namespace slrf {
size_t workspace_estimate(int64_t n, int64_t nnz, int L, int N, int precision, int sm_count, int mg_coarse,
                          int krylov) {
    const size_t Lp = (size_t)(L + 1) / 2 * 2, W = (size_t)N * Lp;
    const size_t ts = precision == SLRF_PREC_MIXED ? 4 : 8;   // Krylov real type
    const size_t gy = std::max<size_t>(1, std::min<size_t>((size_t)(n + 7) / 8, (size_t)sm_count * 8));
    const size_t pencil = (size_t)(n + 1) * 4 + (size_t)nnz * (4 + 8 + 8 + 8 + 16) + (size_t)n * 16 +
                          (size_t)nnz * (4 + 3 * 24) + (size_t)n * 4;
    const size_t kry = 3 * (size_t)n * W * 2 * ts + (size_t)n * N * 2 * ts + (size_t)n * Lp * ts +
                          gy * W * 4 * ts + W * (8 * ts + 40) + 4096;
    const size_t split = (size_t)sm_count * 4;
    const size_t rr = 8 * (size_t)n * L * 8 + split * L * L * 8 + (40 * (size_t)L * L + 64 * (size_t)L) * 8 +
                      (size_t)sm_count * 12 * L * 8 + 8192;
    const size_t ozaki = 2 * 7 * (size_t)((L + 63) / 64 * 64) * (size_t)((n + 63) / 64 * 64) + (size_t)sm_count * 4 * L * L * 8 +
                         ozaki_tall_work_bytes(n, L, L);
    // multigrid (mg_coarse > 0): Z block, level blocks r/z/t and Jacobi
    // diagonals (the levels below the finest hold at most n/2 rows together),
    // transfers and Galerkin pencils (bounded by the fine pattern) and the
    // finest level's fused transfer pairs F (up to ~100 B per stored entry of
    // A), coarsest eigenvectors and shifted inverses
    size_t mgb = 0;
    if (mg_coarse > 0) {
        const size_t nh = (size_t)n / 2 + 1, nc = (size_t)mg_coarse;
        mgb = (size_t)n * W * 2 * ts + 3 * nh * W * 2 * ts + nh * N * 2 * ts + 200 * (size_t)nnz + nc * nc * 12 +
              nc * N * 2 * ts + 16 * 4096 + 768 * 768 * 12 + 768 * (size_t)N * 2 * ts;
        // FP32 cycles ending at a level of at most mg_exact (1536) unknowns: its
        // dense shifted inverses and their elimination work, and (subspace
        // size <= 256) the inverses' bf16 split panels and the per-visit
        // split vectors and partial sums of their tensor-core application
        if (precision == SLRF_PREC_MIXED) {
            const size_t ne = std::min<size_t>(1536, (size_t)n);
            mgb += (size_t)N * ne * ne * 8 + coarse_inverse_work_bytes((int)ne, N);
            if (coarse_tc_fits((int)Lp))
                mgb += coarse_tc_panel_bytes((int)ne, N) + coarse_tc_work_bytes((int)ne, N, (int)Lp);
        }
    }
    // BiCGStab keeps five more n x W blocks (r^, v, y, z, t)
    const size_t bcg = krylov == SLRF_KRYLOV_BICGSTAB ? 5 * (size_t)n * W * 2 * ts + 2 * W * 2 * ts : 0;
    return pencil + kry + rr + ozaki + mgb + bcg;
}
}  // namespace slrf

int slrf::handle_device(const slrf_handle *h) { return h->device; }

// ===========================================================================
// C ABI
// ===========================================================================
namespace {
template <typename T>
slrf_status precond_apply_t(slrf_handle *h, const slrf_filter *f, KrylovDims &d, const cplx<T> *Rb, cplx<T> *Zb,
                            cplx<T> *mu, int32_t *mg_levels) {
    Ctx &ctx = h->ctx;
    const int W = d.W(), N = d.N;
    const int64_t n = d.n;
    KrylovBuffers<T> kb{};
    kb.gy = krylov_row_groups(ctx, d, sizeof(T) == 4);
    *(volatile int32_t *)(h->h_pin + 1) = 0;   // device-side wait timeouts of this solve
    CKS(ensure(h, h->kDinv, (size_t)n * N * sizeof(cplx<T>)));
    CKS(ensure(h, h->kPart, (size_t)kb.gy * W * 4 * sizeof(T)));
    CKS(ensure(h, h->kSig, SLRF_MAX_POLES * sizeof(cplx<T>)));
    CKS(ensure(h, h->kFlags, (size_t)W * 2 * sizeof(int32_t) + 64));
    kb.dinv = as<cplx<T>>(h->kDinv);
    kb.s.part = as<T>(h->kPart);
    kb.s.flag = as<int32_t>(h->kFlags);
    std::vector<int32_t> flags(W);
    for (int col = 0; col < W; ++col) flags[col] = (col % d.Lp) < d.m ? 1 : 0;
    std::vector<cplx<T>> sg(SLRF_MAX_POLES);
    for (int j = 0; j < N; ++j) sg[j] = mk((T)f->sigma_re[j], (T)f->sigma_im[j]);
    CK(cudaMemcpyAsync(kb.s.flag, flags.data(), W * sizeof(int32_t), cudaMemcpyHostToDevice, ctx.stream));
    CK(cudaMemcpyAsync(h->kSig.p, sg.data(), N * sizeof(cplx<T>), cudaMemcpyHostToDevice, ctx.stream));
    const cplx<T> *sig = as<cplx<T>>(h->kSig);
    h->inv_key.clear();
    h->ctx.reset_counters();
    bool use_mg = uses_mg(h);
    if (use_mg) {
        bool usable = true;
        CKS(mg_prepare<T>(h, f, d, kb, h->opts.precond == SLRF_PRECOND_AUTO, &usable));
        use_mg = usable;
    }
    if (use_mg) {
        MgSolve<T> &mg = mg_of<T>(h);
        CKS(ensure(h, h->kQ, (size_t)n * W * sizeof(cplx<T>)));
        mg_apply<T>(ctx, d, mg, sig, kb.s.flag, kb.s.part, kb.gy, Rb, Zb, as<cplx<T>>(h->kQ));
    } else if (h->opts.precond == SLRF_PRECOND_ILU) {
        IluFactor<T> ilu{};
        CKS(ilu_prepare<T>(h, f, d, ilu));
        CKS(ensure(h, h->kQ, (size_t)n * W * sizeof(cplx<T>)));
        ilu_apply<T>(ctx, d, h->ilu_pat, ilu, h->opts.ilu_tri_sweeps, kb.gy, kb.s.flag, Rb, Zb, as<cplx<T>>(h->kQ),
                     as<cplx<T>>(h->kIluY), kb.s.part);
    } else {
        krylov_dinv<T>(ctx, h->A, make_poleset<T>(f),
                       h->opts.precond == SLRF_PRECOND_NONE ? SLRF_PRECOND_NONE : SLRF_PRECOND_JACOBI, kb.dinv);
        bicgstab_precond_jacobi<T>(ctx, d, kb, Rb, Zb);
        mg_rz<T>(ctx, d, kb.gy, Rb, Zb, kb.s.flag, kb.s.part);
    }
    if (mu) krylov_reduce_mu<T>(ctx, d, kb.s.part, kb.gy, mu);
    if (mg_levels) *mg_levels = use_mg ? mg_of<T>(h).nlev : 0;
    CK(cudaStreamSynchronize(ctx.stream));   // the host vectors above are pageable
    CK(cudaGetLastError());
    return SLRF_OK;
}
}  // namespace

extern "C" {

const char *slrf_status_str(slrf_status s) {
    switch (s) {
        case SLRF_OK: return "SLRF_OK";
        case SLRF_EINVAL: return "SLRF_EINVAL";
        case SLRF_ENOMEM: return "SLRF_ENOMEM";
        case SLRF_EBUDGET: return "SLRF_EBUDGET";
        case SLRF_ECUDA: return "SLRF_ECUDA";
        case SLRF_ETIMEOUT: return "SLRF_ETIMEOUT";
        case SLRF_NOT_CONVERGED: return "SLRF_NOT_CONVERGED";
        case SLRF_STAGNATION: return "SLRF_STAGNATION";
        case SLRF_BREAKDOWN: return "SLRF_BREAKDOWN";
        case SLRF_SUBSPACE_TOO_SMALL: return "SLRF_SUBSPACE_TOO_SMALL";
        case SLRF_CHOLQR_FAIL: return "SLRF_CHOLQR_FAIL";
        case SLRF_PENDING: return "SLRF_PENDING";
    }
    return "SLRF_UNKNOWN";
}

const char *slrf_last_error(void) { return g_last_error.c_str(); }

const char *slrf_kernel_class_name(int32_t k) {
    return (k >= 0 && k < SLRF_NKERNEL_CLASSES) ? kKernelClassNames[k] : nullptr;
}

slrf_status slrf_release_cached_memory(int32_t device) {
    cudaMemPool_t pool = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_pool_mu);
        auto it = g_pools.find(device);
        if (it != g_pools.end()) pool = it->second;
    }
    if (!pool) return SLRF_OK;
    CK(cudaMemPoolTrimTo(pool, 0));
    return SLRF_OK;
}

slrf_status slrf_opts_default(slrf_opts *o) {
    if (!o) return SLRF_EINVAL;
    memset(o, 0, sizeof(*o));
    o->precision = SLRF_PREC_MIXED;
    o->krylov = SLRF_KRYLOV_COCG;
    o->precond = SLRF_PRECOND_AUTO;
    o->inner_maxit = 1000;
    o->inner_tol = 1e-5;
    o->lock_tol = 1e-9;
    o->check_every = 4;
    o->eig_refine = 2;
    o->mem_budget = 0;
    o->profile = 0;
    o->spmm_rows = 0;
    o->gram_ozaki = 2;
    o->mg_nu = 0;
    o->mg_cycle = 1;
    o->mg_coarse = 256;
    o->mg_block = 0;
    o->mg_omega = 4.0 / 3.0;
    o->mg_theta = 0.0;
    o->mg_shift_limit = 0.8;
    o->stagnation_window = 8;
    o->mg_exact = 1536;
    o->ilu_sweeps = 3;
    o->ilu_tri_sweeps = 3;
    o->mg_exact_tc = 1;
    o->mg_n_null = 0;
    o->mg_near_null = nullptr;
    return SLRF_OK;
}

static slrf_status check_opts(const slrf_opts *o) {
    if (!o) return SLRF_EINVAL;
    if (o->precision != SLRF_PREC_FP64 && o->precision != SLRF_PREC_MIXED) return SLRF_EINVAL;
    if (o->krylov != SLRF_KRYLOV_COCG && o->krylov != SLRF_KRYLOV_BICGSTAB) return SLRF_EINVAL;
    if (o->precond < SLRF_PRECOND_NONE || o->precond > SLRF_PRECOND_ILU) return SLRF_EINVAL;
    if (o->ilu_sweeps < 0 || o->ilu_sweeps > 32 || o->ilu_tri_sweeps < 1 || o->ilu_tri_sweeps > 32)
        return SLRF_EINVAL;
    if (o->mg_nu < 0 || o->mg_nu > 8 || o->mg_cycle < 1 || o->mg_cycle > 2 || o->mg_coarse < 1 ||
        o->mg_coarse > 4096 || o->mg_block < 0 || o->mg_block > 8 || !(o->mg_omega > 0.0) ||
        !(o->mg_omega < 2.0) || !(o->mg_theta >= 0.0) || !(o->mg_theta < 1.0) || o->stagnation_window < 0 ||
        !(o->mg_shift_limit > 0.0))
        return SLRF_EINVAL;
    if (o->inner_maxit < 1 || !(o->inner_tol > 0) || o->check_every < 1 || o->mem_budget < 0) return SLRF_EINVAL;
    if (o->spmm_rows < 0 || o->spmm_rows > 4) return SLRF_EINVAL;
    if (o->spmm_kernel < 0 || o->spmm_kernel > 4) return SLRF_EINVAL;
    if (o->eig_refine < 0 || o->eig_refine > 2) return SLRF_EINVAL;
    if (o->mg_exact_tc < 0 || o->mg_exact_tc > 1) return SLRF_EINVAL;
    if (o->mg_n_null < 0 || o->mg_n_null > 16 || (o->mg_n_null > 0 && !o->mg_near_null)) return SLRF_EINVAL;
    if (o->sell_c != 0 && o->sell_c != 4 && o->sell_c != 8 && o->sell_c != 16 && o->sell_c != 32 && o->sell_c != 64)
        return SLRF_EINVAL;
    if (o->sell_sigma < 0) return SLRF_EINVAL;
    if (o->gram_ozaki < 0 || o->gram_ozaki > 2) return SLRF_EINVAL;
    if (o->mg_exact < 0 || o->mg_exact > 4096) return SLRF_EINVAL;
    return SLRF_OK;
}

slrf_status slrf_mg_describe(const slrf_pencil *p, const slrf_opts *o, int32_t *n_levels, int64_t *level_n,
                             int64_t *level_nnz, double *setup_ms, double *coarse_lam, double *coarse_a,
                             double *coarse_b) {
    if (!p || p->on_device || !n_levels || !level_n || !level_nnz) return SLRF_EINVAL;
    if (p->n < 1 || p->n > (1LL << 31) - 2 || p->nnz < p->n || p->nnz > (1LL << 31) - 1 || !p->row_ptr ||
        !p->col_idx || !p->a_val || !p->b_val)
        return SLRF_EINVAL;
    slrf_opts def;
    slrf_opts_default(&def);
    if (!o) o = &def;
    CKS(check_opts(o));
    const int64_t n = p->n, nnz = p->nnz;
    std::vector<int32_t> rp(p->row_ptr, p->row_ptr + n + 1), ci(p->col_idx, p->col_idx + nnz);
    std::vector<double> av(p->a_val, p->a_val + nnz), bv(p->b_val, p->b_val + nnz);
    if (!pencil_valid(n, nnz, rp, ci, av, bv)) return SLRF_EINVAL;
    std::vector<double> nul;
    if (!copy_near_null(*o, n, nul)) return SLRF_EINVAL;
    const int block = mg_block_for(*o, n, rp, ci);
    MgParams prm = mg_params(*o, block);
    prm.near_null = nul.empty() ? nullptr : nul.data();
    prm.n_null = nul.empty() ? 0 : o->mg_n_null;
    HostHierarchy H;
    const std::string err = mg_build((int)n, rp.data(), ci.data(), av.data(), bv.data(), prm, H);
    if (!err.empty()) {
        g_last_error = err;
        return SLRF_BREAKDOWN;
    }
    const int nlev = (int)H.lv.size();
    if (nlev > SLRF_MG_MAX_LEVELS) return SLRF_BREAKDOWN;
    *n_levels = nlev;
    for (int l = 0; l < nlev; ++l) {
        level_n[l] = H.lv[l].n;
        level_nnz[l] = l == 0 ? nnz : (int64_t)H.lv[l].col.size();
    }
    if (setup_ms) *setup_ms = H.ms_setup;
    const HostLevel &Lc = H.lv.back();
    const int nc = Lc.n;
    if (coarse_lam) std::copy(H.lam.begin(), H.lam.end(), coarse_lam);
    if (coarse_a || coarse_b) {
        const int32_t *cp = nlev == 1 ? rp.data() : Lc.ptr.data();
        const int32_t *cc = nlev == 1 ? ci.data() : Lc.col.data();
        const double *ca = nlev == 1 ? av.data() : Lc.a.data();
        const double *cb = nlev == 1 ? bv.data() : Lc.b.data();
        if (coarse_a) std::fill(coarse_a, coarse_a + (size_t)nc * nc, 0.0);
        if (coarse_b) std::fill(coarse_b, coarse_b + (size_t)nc * nc, 0.0);
        for (int i = 0; i < nc; ++i)
            for (int32_t k = cp[i]; k < cp[i + 1]; ++k) {
                if (coarse_a) coarse_a[(size_t)i * nc + cc[k]] = ca[k];
                if (coarse_b) coarse_b[(size_t)i * nc + cc[k]] = cb[k];
            }
    }
    return SLRF_OK;
}

slrf_status slrf_mg_transfer(const slrf_pencil *p, const slrf_opts *o, int32_t level, int32_t *n_rows,
                             int32_t *n_cols, int64_t *nnz, double *rho, int32_t *ptr, int32_t *col, double *val) {
    if (!p || p->on_device || !n_rows || !n_cols || !nnz || !rho || level < 0) return SLRF_EINVAL;
    if (p->n < 1 || p->n > (1LL << 31) - 2 || p->nnz < p->n || p->nnz > (1LL << 31) - 1 || !p->row_ptr ||
        !p->col_idx || !p->a_val || !p->b_val)
        return SLRF_EINVAL;
    slrf_opts def;
    slrf_opts_default(&def);
    if (!o) o = &def;
    CKS(check_opts(o));
    const int64_t n = p->n, nnzA = p->nnz;
    std::vector<int32_t> rp(p->row_ptr, p->row_ptr + n + 1), ci(p->col_idx, p->col_idx + nnzA);
    std::vector<double> av(p->a_val, p->a_val + nnzA), bv(p->b_val, p->b_val + nnzA);
    if (!pencil_valid(n, nnzA, rp, ci, av, bv)) return SLRF_EINVAL;
    std::vector<double> nul;
    if (!copy_near_null(*o, n, nul)) return SLRF_EINVAL;
    MgParams prm = mg_params(*o, mg_block_for(*o, n, rp, ci));
    prm.near_null = nul.empty() ? nullptr : nul.data();
    prm.n_null = nul.empty() ? 0 : o->mg_n_null;
    HostHierarchy H;
    const std::string err = mg_build((int)n, rp.data(), ci.data(), av.data(), bv.data(), prm, H);
    if (!err.empty()) {
        g_last_error = err;
        return SLRF_BREAKDOWN;
    }
    if (level > (int)H.lv.size() - 2) return SLRF_EINVAL;
    const HostCsr &P = H.lv[level].P;
    *n_rows = P.n_rows;
    *n_cols = P.n_cols;
    *nnz = (int64_t)P.col.size();
    *rho = H.lv[level].rho;
    if (ptr) std::copy(P.ptr.begin(), P.ptr.end(), ptr);
    if (col) std::copy(P.col.begin(), P.col.end(), col);
    if (val) std::copy(P.val.begin(), P.val.end(), val);
    return SLRF_OK;
}

slrf_status slrf_set_opts(slrf_handle *h, const slrf_opts *o) {
    if (!h) return SLRF_EINVAL;
    CKS(check_opts(o));
    std::vector<double> nul;
    if (!copy_near_null(*o, h->A.n, nul)) return SLRF_EINVAL;
    const int k = nul.empty() ? 0 : o->mg_n_null;
    if (k != h->mg_null_k || nul != h->mg_null) {
        h->mg_null.swap(nul);
        h->mg_null_k = k;
        h->mg_null_dirty = true;
    }
    h->opts = *o;
    h->opts.mg_near_null = nullptr;   // the handle keeps its own copy
    h->ctx.profile = o->profile != 0;
    h->ctx.profile_mask = o->profile_mask ? o->profile_mask : ~0u;
    h->A.spmm_kind = o->spmm_kernel;
    return SLRF_OK;
}

void slrf_destroy(slrf_handle *h) {
    if (!h) return;
    Buf *bufs[] = {&h->kP, &h->kQ, &h->kR, &h->kDinv, &h->kU, &h->kPart, &h->kSig, &h->kScal, &h->kFlags,
                   &h->rOz, &h->rW1, &h->rQ1, &h->rQ2, &h->rX, &h->rAX, &h->rBX, &h->rRes, &h->rSmall, &h->rSplit, &h->rV,
                   &h->rTheta, &h->rRho, &h->hostV, &h->hostX, &h->mgStatic, &h->mgState, &h->kZ, &h->rOzT, &h->kBcg, &h->rTallB,
                   &h->mgInvPan, &h->mgCtWork,
                   &h->mg_eig[0].dev, &h->mg_eig[1].dev, &h->mg_eig[2].dev, &h->mg_eig[3].dev,
                   &h->mg_eig[4].dev, &h->mg_eig[5].dev, &h->mg_eig[6].dev, &h->mg_eig[7].dev,
                   &h->mg_eig[8].dev, &h->mg_eig[9].dev, &h->mg_eig[10].dev, &h->mg_eig[11].dev,
                   &h->mg_eig[12].dev, &h->mg_eig[13].dev, &h->mg_eig[14].dev, &h->mg_eig[15].dev};
    for (Buf *b : bufs)
        if (b->p) cudaFreeAsync(b->p, h->ctx.stream);
    if (h->mgInv.p) cudaFreeAsync(h->mgInv.p, h->ctx.stream);
    for (Buf *b : {&h->iluPat, &h->iluFac, &h->kIluY})
        if (b->p) cudaFreeAsync(b->p, h->ctx.stream);
    if (h->cublas) cublasDestroy(h->cublas);
    void *pen[] = {h->A.rowptr, h->A.col,    h->A.a,      h->A.b,       h->A.ab32,   h->A.ab64,
                   h->A.diag_a, h->A.diag_b, h->A.rg_ptr, h->A.rg_col, h->A.rg_ab32, h->A.rg_ab64,
                   h->A.rg_ab4, h->A.rg_dpos, h->A.nb_ptr, h->A.nb_node, h->A.nb_coef,
                   h->A.sell_cptr, h->A.sell_col, h->A.sell_ab, h->A.sell_perm, h->A.sell_rlen};
    for (void *p : pen)
        if (p) cudaFreeAsync(p, h->ctx.stream);
    cudaStreamSynchronize(h->ctx.stream);
    if (h->h_pin) pin_release(h->h_pin);
    if (h->ev_poll) cudaEventDestroy(h->ev_poll);
    if (h->ev_t0) cudaEventDestroy(h->ev_t0);
    if (h->ev_t1) cudaEventDestroy(h->ev_t1);
    for (auto &e : h->phase_k) {
        cudaEventDestroy(e.first);
        cudaEventDestroy(e.second);
    }
    for (auto &e : h->phase_r) {
        cudaEventDestroy(e.first);
        cudaEventDestroy(e.second);
    }
    h->ctx.destroy();
    delete h;
}

slrf_status slrf_create(slrf_handle **out, const slrf_pencil *p, const slrf_opts *o, void *cuda_stream) {
    if (!out) return SLRF_EINVAL;
    *out = nullptr;
    if (!p || p->n < 1 || p->n > (1LL << 31) - 2 || p->nnz < p->n || p->nnz > (1LL << 31) - 1 || !p->row_ptr ||
        !p->col_idx || !p->a_val || !p->b_val)
        return SLRF_EINVAL;
    slrf_opts def;
    slrf_opts_default(&def);
    if (!o) o = &def;
    CKS(check_opts(o));
    const int64_t n = p->n, nnz = p->nnz;
    // host copies for validation (shared with the multigrid setup thread,
    // which may outlive this call)
    struct HostCopy {
        std::vector<int32_t> rp, ci;
        std::vector<double> av, bv;
        std::vector<double> nul;   // the options' near-null space
    };
    auto hc = std::make_shared<HostCopy>();
    std::vector<int32_t> &rp = hc->rp, &ci = hc->ci;
    std::vector<double> &av = hc->av, &bv = hc->bv;
    if (p->on_device) {
        rp.resize(n + 1);
        ci.resize(nnz);
        av.resize(nnz);
        bv.resize(nnz);
        CK(cudaMemcpy(rp.data(), p->row_ptr, (n + 1) * sizeof(int32_t), cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(ci.data(), p->col_idx, nnz * sizeof(int32_t), cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(av.data(), p->a_val, nnz * sizeof(double), cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(bv.data(), p->b_val, nnz * sizeof(double), cudaMemcpyDeviceToHost));
    } else {   // the four arrays copied side by side
        host_team(4, [&](int t) {
            if (t == 0) rp.assign(p->row_ptr, p->row_ptr + n + 1);
            if (t == 1) ci.assign(p->col_idx, p->col_idx + nnz);
            if (t == 2) av.assign(p->a_val, p->a_val + nnz);
            if (t == 3) bv.assign(p->b_val, p->b_val + nnz);
        });
    }
    if (!pencil_valid(n, nnz, rp, ci, av, bv)) return SLRF_EINVAL;
    if (!copy_near_null(*o, n, hc->nul)) return SLRF_EINVAL;
    // Row grouping of the shifted SpMM (measured on the 2D Q1 pencil: 2 rows
    // per group beats 1 and 4; 3-dof elasticity groups the rows of a node).
    const bool blocks = has_node_blocks(n, rp, ci, 3);
    int R = o->spmm_rows;
    if (R == 0) R = blocks ? 3 : 2;
    // The multigrid hierarchy (host) is built, and its device image laid out,
    // on its own thread while the pencil is uploaded and its row-group form
    // built on the device; the handle keeps the pending result, and the first solve
    // that needs the hierarchy waits for it (after the work it can do
    // without it, such as the first projection of the start block).
    slrf_opts opts_copy = *o;
    opts_copy.mg_near_null = nullptr;   // the setup thread reads hc->nul
    const bool want_mg = o->precond == SLRF_PRECOND_MG || (o->precond == SLRF_PRECOND_AUTO && !blocks);
    const int mg_blk = want_mg ? mg_block_for(opts_copy, n, rp, ci) : 0;
    struct MgBuilt {
        std::string err;
        std::shared_ptr<HostHierarchy> H;
        MgStaged S;
        std::shared_future<std::string> eig;   // coarsest eigenpairs, if still running
    };
    std::future<MgBuilt> mg_fut;
    auto build_mg = [hc, opts_copy, n, mg_blk, R] {
        MgBuilt r;
        r.H = std::make_shared<HostHierarchy>();
        MgParams prm = mg_params(opts_copy, mg_blk);
        prm.defer_coarse_eig = true;
        prm.near_null = hc->nul.empty() ? nullptr : hc->nul.data();
        prm.n_null = hc->nul.empty() ? 0 : opts_copy.mg_n_null;
        r.err = mg_build((int)n, hc->rp.data(), hc->ci.data(), hc->av.data(), hc->bv.data(), prm, *r.H);
        if (!r.err.empty()) return r;
        // the coarsest level's eigenpairs on a thread of their own: a cycle
        // that ends at a level with dense shifted inverses never needs them,
        // and the first one that does waits for them
        try {
            r.eig = std::async(std::launch::async, [Hp = r.H] { return mg_coarse_eig(*Hp); }).share();
        } catch (...) {   // no thread: in line
        }
        mg_stage(*r.H, R > 1 ? R : 1, r.S);
        if (!r.eig.valid()) {
            r.err = mg_coarse_eig(*r.H);
            if (r.err.empty()) mg_stage_v(*r.H, r.S);
        }
        return r;
    };
    if (want_mg) {
        try {
            mg_fut = std::async(std::launch::async, build_mg);
        } catch (...) {   // no thread: built synchronously below
        }
    }
    slrf_handle *h = new slrf_handle();
    h->opts = *o;
    h->opts.mg_near_null = nullptr;   // the handle keeps its own copy
    h->mg_null = hc->nul;
    h->mg_null_k = hc->nul.empty() ? 0 : o->mg_n_null;
    h->node_blocks = blocks;
    h->ctx.stream = reinterpret_cast<cudaStream_t>(cuda_stream);
    h->ctx.profile = o->profile != 0;
    h->ctx.profile_mask = o->profile_mask ? o->profile_mask : ~0u;
    cudaGetDevice(&h->device);
    cudaDeviceGetAttribute(&h->ctx.sm_count, cudaDevAttrMultiProcessorCount, h->device);
    h->A.n = (int)n;
    h->A.nnz = nnz;
    const size_t need = (n + 1) * 4 + nnz * (4 + 8 + 8 + 8 + 16) + n * 16;
    if (o->mem_budget > 0 && need > (size_t)o->mem_budget) {
        delete h;
        return SLRF_EBUDGET;
    }
    auto alloc = [&](void **ptr, size_t bytes) -> bool {
        if (dev_alloc(h, ptr, bytes) != cudaSuccess) {
            *ptr = nullptr;
            cudaGetLastError();
            return false;
        }
        h->pencil_bytes += bytes;
        return true;
    };
    bool ok = alloc((void **)&h->A.rowptr, (n + 1) * 4) && alloc((void **)&h->A.col, nnz * 4) &&
              alloc((void **)&h->A.a, nnz * 8) && alloc((void **)&h->A.b, nnz * 8) &&
              alloc((void **)&h->A.ab32, nnz * 8) && alloc((void **)&h->A.ab64, nnz * 16) &&
              alloc((void **)&h->A.diag_a, n * 8) && alloc((void **)&h->A.diag_b, n * 8) &&
              pin_acquire(&h->h_pin, &h->d_pin);
    if (!ok) {
        g_last_error = "device allocation of the pencil failed";
        slrf_destroy(h);
        return SLRF_ENOMEM;
    }
    h->A.dev_err = h->d_pin + 1;   // second word of the handle's pinned poll slot
    h->A.spmm_kind = o->spmm_kernel;
    cudaEventCreate(&h->ev_poll);
    cudaEventCreate(&h->ev_t0);
    cudaEventCreate(&h->ev_t1);
    cudaStream_t s = h->ctx.stream;
    // from the caller's arrays (pinned host memory or device memory is read
    // directly); complete before this call returns
    cudaMemcpyAsync(h->A.rowptr, p->row_ptr, (n + 1) * 4, cudaMemcpyDefault, s);
    cudaMemcpyAsync(h->A.col, p->col_idx, nnz * 4, cudaMemcpyDefault, s);
    cudaMemcpyAsync(h->A.a, p->a_val, nnz * 8, cudaMemcpyDefault, s);
    cudaMemcpyAsync(h->A.b, p->b_val, nnz * 8, cudaMemcpyDefault, s);
    k_pack_ab<<<(unsigned)((nnz + 255) / 256), 256, 0, s>>>(nnz, h->A.a, h->A.b, h->A.ab32, h->A.ab64);
    k_diag<<<(unsigned)((n + 255) / 256), 256, 0, s>>>((int)n, h->A.rowptr, h->A.col, h->A.a, h->A.b, h->A.diag_a,
                                                         h->A.diag_b);
    if (R > 1) {
        // row-group form, built on the device from the uploaded CSR: sizes
        // (one merge per group), prefix sum and largest group, then the arrays
        const int64_t ng = (n + R - 1) / R;
        if (!alloc((void **)&h->A.rg_ptr, (ng + 2) * 4)) {
            g_last_error = "device allocation of the row-group pencil failed";
            slrf_destroy(h);
            return SLRF_ENOMEM;
        }
        const unsigned gb = (unsigned)((ng + 255) / 256);
        k_rg_count<<<gb, 256, 0, s>>>(n, R, ng, h->A.rowptr, h->A.col, h->A.rg_ptr);
        k_rg_scan<<<1, 1024, 0, s>>>(ng, h->A.rg_ptr, h->A.rg_ptr + ng + 1);
        int32_t tail[2] = {0, 0};   // union entries, largest group
        cudaMemcpyAsync(tail, h->A.rg_ptr + ng, sizeof(tail), cudaMemcpyDeviceToHost, s);
        const cudaError_t e0 = cudaStreamSynchronize(s);
        if (e0 != cudaSuccess) {
            g_last_error = std::string("pencil upload: ") + cudaGetErrorString(e0);
            slrf_destroy(h);
            return SLRF_ECUDA;
        }
        const int64_t U = tail[0];
        if (!(alloc((void **)&h->A.rg_col, U * 4) && alloc((void **)&h->A.rg_ab32, U * R * 8) &&
              alloc((void **)&h->A.rg_ab64, U * R * 16))) {
            g_last_error = "device allocation of the row-group pencil failed";
            slrf_destroy(h);
            return SLRF_ENOMEM;
        }
        h->A.rg_rows = R;
        h->A.rg_ngroups = (int)ng;
        h->A.rg_nnz = U;
        h->A.rg_emax = tail[1];
        // staged-kernel form, optional (without it the row-group kernel
        // runs): packed (a, a, b, b) pairs and own-column positions
        if (tail[1] <= 255 && !(alloc((void **)&h->A.rg_ab4, U * R * 16) && alloc((void **)&h->A.rg_dpos, ng * R))) {
            for (void **q : {(void **)&h->A.rg_ab4, (void **)&h->A.rg_dpos})
                if (*q) {
                    cudaFreeAsync(*q, s);
                    *q = nullptr;
                }
        }
        k_rg_fill<<<gb, 256, 0, s>>>(n, R, ng, h->A.rowptr, h->A.col, h->A.a, h->A.b, h->A.rg_ptr, h->A.rg_col,
                                     h->A.rg_ab32, h->A.rg_ab64, h->A.rg_ab4, h->A.rg_dpos);
        // node-block form (optional: without it the row-group kernel runs)
        std::vector<int32_t> nptr, nnode;
        std::vector<float4> ncoef;
        if (R == 3 && build_nodeblocks(n, rp, ci, av, bv, nptr, nnode, ncoef) &&
            alloc((void **)&h->A.nb_ptr, nptr.size() * 4) && alloc((void **)&h->A.nb_node, nnode.size() * 4) &&
            alloc((void **)&h->A.nb_coef, ncoef.size() * 16)) {
            cudaMemcpyAsync(h->A.nb_ptr, nptr.data(), nptr.size() * 4, cudaMemcpyHostToDevice, s);
            cudaMemcpyAsync(h->A.nb_node, nnode.data(), nnode.size() * 4, cudaMemcpyHostToDevice, s);
            cudaMemcpyAsync(h->A.nb_coef, ncoef.data(), ncoef.size() * 16, cudaMemcpyHostToDevice, s);
            cudaStreamSynchronize(s);   // pageable sources
        } else {
            for (void **q : {(void **)&h->A.nb_ptr, (void **)&h->A.nb_node, (void **)&h->A.nb_coef})
                if (*q) {
                    cudaFreeAsync(*q, s);
                    *q = nullptr;
                }
        }
    }
    // SELL-C-sigma form: built here when asked for, else when the kernel
    // autotuner first times it for this pattern (from the device copy)
    if (o->spmm_kernel == SPMM_SELL) {
        const slrf_status st = sell_upload(h, rp, ci, av, bv);
        if (st != SLRF_OK) {
            slrf_destroy(h);
            return st;
        }
    }
    const cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        g_last_error = std::string("pencil upload: ") + cudaGetErrorString(e);
        slrf_destroy(h);
        return SLRF_ECUDA;
    }
    if (want_mg) {
        auto finish = [mg_blk](slrf_handle *hh, MgBuilt built) -> slrf_status {
            if (!built.err.empty()) {
                g_last_error = built.err;
                return SLRF_BREAKDOWN;
            }
            return mg_upload(hh, *built.H, built.S, mg_blk, built.H, built.eig);
        };
        if (mg_fut.valid()) {
            auto fut = std::make_shared<std::future<MgBuilt>>(std::move(mg_fut));
            h->mg_finish = [fut, finish](slrf_handle *hh) -> slrf_status {
                MgBuilt built;
                try {
                    built = fut->get();
                } catch (const std::exception &ex) {
                    built.err = std::string("multigrid setup: ") + ex.what();
                }
                return finish(hh, std::move(built));
            };
        } else {   // no setup thread: built here
            const slrf_status st = finish(h, build_mg());
            if (st != SLRF_OK) {
                slrf_destroy(h);
                return st;
            }
        }
    }
    *out = h;
    return SLRF_OK;
}


slrf_status slrf_filter_apply(slrf_handle *h, const slrf_filter *f, const double *V, int64_t ldv, int32_t m,
                              double *U, int64_t ldu, slrf_report *rep) {
    if (!h) return SLRF_EINVAL;
    CKS(check_filter(f));
    CKS(check_dense(V, ldv, m));
    CKS(check_dense(U, ldu, m));
    CallScope scope(h, rep);
    Ctx &ctx = h->ctx;
    const int64_t n = h->A.n;
    const int N = f->n_poles;
    CKS(ensure(h, h->rBX, (size_t)n * m * sizeof(double)));
    double *F = as<double>(h->rBX);
    spmm_real(ctx, h->A, m, V, ldv, nullptr, 0, F, m);
    std::vector<int> active(m, 1);
    std::vector<cd> coef((size_t)N * m);
    for (int j = 0; j < N; ++j)
        for (int c = 0; c < m; ++c) coef[(size_t)j * m + c] = cd(f->w_re[j], f->w_im[j]);
    KrylovDims d;
    KStats st;
    slrf_status s;
    phase_begin(h, h->phase_k, h->phase_k_used);
    if (h->opts.precision == SLRF_PREC_MIXED) {
        KrylovBuffers<float> kb;
        s = krylov_solve<float>(h, f, m, F, m, active, coef, h->opts.inner_tol, h->opts.inner_maxit, kb, d, st);
        if (s == SLRF_OK) filter_combine<float>(ctx, (int)n, m, nullptr, 0, nullptr, kb.Uacc, d.Lp, U, ldu);
    } else {
        KrylovBuffers<double> kb;
        s = krylov_solve<double>(h, f, m, F, m, active, coef, h->opts.inner_tol, h->opts.inner_maxit, kb, d, st);
        if (s == SLRF_OK) filter_combine<double>(ctx, (int)n, m, nullptr, 0, nullptr, kb.Uacc, d.Lp, U, ldu);
    }
    phase_end(h, h->phase_k, h->phase_k_used);
    if (s != SLRF_OK) return s;
    if (rep) {
        rep->outer_iters = 1;
        rep->krylov_iters = st.iters_max;
        rep->spmv = st.spmv;
        for (int j = 0; j < N; ++j) rep->iters_per_pole[j] = st.iters_per_pole[j];
        rep->status_detail = st.n_fail + st.n_breakdown;
        rep->mg_levels = st.mg_levels;
        rep->spmm_kernel = h->A.spmm_kind;
    }
    scope.finish();
    CK(cudaGetLastError());
    return (st.n_fail + st.n_breakdown) ? SLRF_NOT_CONVERGED : SLRF_OK;
}

slrf_status slrf_subspace_iterate(slrf_handle *h, const slrf_filter *f, double gamma, int32_t L, const double *V0,
                                  int64_t ldv, double tol, int32_t max_outer, double *theta, double *X, int64_t ldx,
                                  double *resid, int32_t *n_conv, slrf_report *rep) {
    if (!h || !(gamma > 0) || !(tol > 0) || max_outer < 1 || !theta || !resid) return SLRF_EINVAL;
    CKS(check_filter(f));
    CKS(check_dense(V0, ldv, L));
    CKS(check_dense(X, ldx, L));
    if (L > h->A.n || L > 1024) return SLRF_EINVAL;
    CallScope scope(h, rep);
    const slrf_status s = subspace_core(h, f, gamma, L, V0, ldv, tol, max_outer, theta, X, ldx, resid, n_conv, rep);
    scope.finish();
    if (s == SLRF_ECUDA || s == SLRF_ENOMEM || s == SLRF_EBUDGET) return s;
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        g_last_error = cudaGetErrorString(e);
        return SLRF_ECUDA;
    }
    return s;
}

// Copies between a contiguous device block (rows x width bytes) and a host
// block of row pitch ldh bytes.  A pitched copy to or from pageable host
// memory runs row by row in the driver (measured ~90 ms for 89 401 rows of
// 1.2 KB on GB300, against ~4 ms for one contiguous copy), so a pitched
// pageable host block goes through one contiguous copy and a host-side row
// gather or scatter; pinned host blocks keep the pitched DMA copy.
static bool host_is_pinned(const void *p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeHost;
}

static cudaError_t copy_rows_h2d(void *dev, const void *host, size_t ldh, size_t width, size_t rows, cudaStream_t s) {
    if (ldh == width) return cudaMemcpyAsync(dev, host, width * rows, cudaMemcpyHostToDevice, s);
    if (host_is_pinned(host)) return cudaMemcpy2DAsync(dev, width, host, ldh, width, rows, cudaMemcpyHostToDevice, s);
    std::vector<char> tmp(width * rows);
    for (size_t r = 0; r < rows; ++r) memcpy(tmp.data() + r * width, (const char *)host + r * ldh, width);
    const cudaError_t e = cudaMemcpyAsync(dev, tmp.data(), width * rows, cudaMemcpyHostToDevice, s);
    return e != cudaSuccess ? e : cudaStreamSynchronize(s);
}

static cudaError_t copy_rows_d2h(void *host, size_t ldh, const void *dev, size_t width, size_t rows, cudaStream_t s) {
    if (ldh == width) return cudaMemcpyAsync(host, dev, width * rows, cudaMemcpyDeviceToHost, s);
    if (host_is_pinned(host)) return cudaMemcpy2DAsync(host, ldh, dev, width, width, rows, cudaMemcpyDeviceToHost, s);
    std::vector<char> tmp(width * rows);
    cudaError_t e = cudaMemcpyAsync(tmp.data(), dev, width * rows, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    for (size_t r = 0; r < rows; ++r) memcpy((char *)host + r * ldh, tmp.data() + r * width, width);
    return cudaSuccess;
}

slrf_status slrf_subspace_iterate_host(slrf_handle *h, const slrf_filter *f, double gamma, int32_t L,
                                       const double *V0, int64_t ldv, double tol, int32_t max_outer, double *theta,
                                       double *X, int64_t ldx, double *resid, int32_t *n_conv, slrf_report *rep) {
    if (!h || !V0 || !X || !theta || !resid || L < 1 || ldv < L || ldx < L) return SLRF_EINVAL;
    const int64_t n = h->A.n;
    CKS(ensure(h, h->hostV, (size_t)n * L * sizeof(double)));
    CKS(ensure(h, h->hostX, (size_t)n * L * sizeof(double) + 2 * (size_t)L * sizeof(double)));
    double *dV = as<double>(h->hostV), *dX = as<double>(h->hostX);
    double *dth = dX + (size_t)n * L, *dres = dth + L;
    cudaStream_t s = h->ctx.stream;
    CK(copy_rows_h2d(dV, V0, (size_t)ldv * 8, (size_t)L * 8, (size_t)n, s));
    const slrf_status st = slrf_subspace_iterate(h, f, gamma, L, dV, L, tol, max_outer, dth, dX, L, dres, n_conv, rep);
    if (st == SLRF_EINVAL || st == SLRF_ECUDA || st == SLRF_ENOMEM || st == SLRF_EBUDGET) return st;
    CK(copy_rows_d2h(X, (size_t)ldx * 8, dX, (size_t)L * 8, (size_t)n, s));
    CK(cudaMemcpyAsync(theta, dth, L * 8, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(resid, dres, L * 8, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return st;
}

slrf_status slrf_shifted_spmm(slrf_handle *h, const slrf_filter *f, int32_t prec, int32_t m, int32_t ldp,
                              const void *P, void *Q, void *mu) {
    if (!h || !P || !Q || m < 1 || ldp < m || (ldp & 1)) return SLRF_EINVAL;
    CKS(check_filter(f));
    Ctx &ctx = h->ctx;
    KrylovDims d;
    d.n = h->A.n;
    d.N = f->n_poles;
    d.Lp = ldp;
    d.m = m;
    const int W = d.W();
    const int gy = krylov_row_groups(ctx, d, prec == SLRF_PREC_MIXED);
    const size_t esz = prec == SLRF_PREC_MIXED ? sizeof(float) : sizeof(double);
    CKS(ensure(h, h->kPart, (size_t)gy * W * 4 * esz));
    CKS(ensure(h, h->kSig, SLRF_MAX_POLES * 2 * esz));
    CKS(ensure(h, h->kFlags, (size_t)W * 2 * sizeof(int32_t) + 64));
    std::vector<int32_t> flags(W);
    for (int col = 0; col < W; ++col) flags[col] = (col % ldp) < m ? 1 : 0;
    CK(cudaMemcpyAsync(h->kFlags.p, flags.data(), W * 4, cudaMemcpyHostToDevice, ctx.stream));
    h->ctx.reset_counters();
    CK(cudaStreamSynchronize(ctx.stream));
    *(volatile int32_t *)(h->h_pin + 1) = 0;
    if (prec == SLRF_PREC_MIXED) {
        std::vector<float2> sg(d.N);
        for (int j = 0; j < d.N; ++j) sg[j] = make_float2((float)f->sigma_re[j], (float)f->sigma_im[j]);
        CK(cudaMemcpyAsync(h->kSig.p, sg.data(), d.N * sizeof(float2), cudaMemcpyHostToDevice, ctx.stream));
        krylov_spmm<float>(ctx, d, h->A, as<float2>(h->kSig), (const float2 *)P, (float2 *)Q, as<int32_t>(h->kFlags),
                           as<float>(h->kPart), gy);
        if (mu) krylov_reduce_mu<float>(ctx, d, as<float>(h->kPart), gy, (float2 *)mu);
    } else if (prec == SLRF_PREC_FP64) {
        std::vector<double2> sg(d.N);
        for (int j = 0; j < d.N; ++j) sg[j] = make_double2(f->sigma_re[j], f->sigma_im[j]);
        CK(cudaMemcpyAsync(h->kSig.p, sg.data(), d.N * sizeof(double2), cudaMemcpyHostToDevice, ctx.stream));
        krylov_spmm<double>(ctx, d, h->A, as<double2>(h->kSig), (const double2 *)P, (double2 *)Q,
                            as<int32_t>(h->kFlags), as<double>(h->kPart), gy);
        if (mu) krylov_reduce_mu<double>(ctx, d, as<double>(h->kPart), gy, (double2 *)mu);
    } else {
        return SLRF_EINVAL;
    }
    CK(cudaStreamSynchronize(ctx.stream));
    CK(cudaGetLastError());
    if (*(volatile int32_t *)(h->h_pin + 1) != 0) {
        g_last_error = "shifted product: a bounded device wait gave up";
        return SLRF_ETIMEOUT;
    }
    return SLRF_OK;
}

slrf_status slrf_precond_apply(slrf_handle *h, const slrf_filter *f, int32_t prec, int32_t m, int32_t ldp,
                               const void *R, void *Z, void *mu, int32_t *mg_levels) {
    if (!h || !R || !Z || m < 1 || ldp < m || (ldp & 1)) return SLRF_EINVAL;
    CKS(check_filter(f));
    KrylovDims d;
    d.n = h->A.n;
    d.N = f->n_poles;
    d.Lp = ldp;
    d.m = m;
    if (prec == SLRF_PREC_MIXED)
        return precond_apply_t<float>(h, f, d, (const float2 *)R, (float2 *)Z, (float2 *)mu, mg_levels);
    if (prec == SLRF_PREC_FP64)
        return precond_apply_t<double>(h, f, d, (const double2 *)R, (double2 *)Z, (double2 *)mu, mg_levels);
    return SLRF_EINVAL;
}

slrf_status slrf_spmm_ab(slrf_handle *h, int32_t m, const double *X, int64_t ldx, double *Y, int64_t ldy, double *Z,
                         int64_t ldz) {
    if (!h || !X || m < 1 || ldx < m || (Y && ldy < m) || (Z && ldz < m) || (!Y && !Z)) return SLRF_EINVAL;
    spmm_real(h->ctx, h->A, m, X, ldx, Y, ldy, Z, ldz);
    CK(cudaGetLastError());
    return SLRF_OK;
}

slrf_status slrf_gram(slrf_handle *h, int32_t m, const double *X, int64_t ldx, const double *Y, int64_t ldy,
                      double *G) {
    if (!h || !X || !Y || !G || m < 1 || ldx < m || ldy < m) return SLRF_EINVAL;
    CK(cudaStreamSynchronize(h->ctx.stream));
    *(volatile int32_t *)(h->h_pin + 1) = 0;
    CKS(gram(h, h->A.n, m, X, ldx, Y, ldy, G));
    CK(cudaStreamSynchronize(h->ctx.stream));
    CK(cudaGetLastError());
    if (*(volatile int32_t *)(h->h_pin + 1) != 0) {
        g_last_error = "Gram: a bounded device wait gave up";
        return SLRF_ETIMEOUT;
    }
    return SLRF_OK;
}

slrf_status slrf_tall_product(slrf_handle *h, int32_t k, int32_t m, const double *A, int64_t lda, const double *B,
                              int64_t ldb, double *C, int64_t ldc) {
    if (!h || !A || !B || !C || k < 1 || m < 1 || lda < k || ldb < m || ldc < m) return SLRF_EINVAL;
    CK(cudaStreamSynchronize(h->ctx.stream));
    *(volatile int32_t *)(h->h_pin + 1) = 0;
    CKS(ensure(h, h->rTallB, (size_t)k * m * sizeof(double)));
    // tall_product may scale B in place (FP64 path with column scaling): a copy
    CK(cudaMemcpy2DAsync(h->rTallB.p, (size_t)m * 8, B, (size_t)ldb * 8, (size_t)m * 8, (size_t)k,
                         cudaMemcpyDeviceToDevice, h->ctx.stream));
    CKS(tall_product(h, h->A.n, k, m, A, lda, nullptr, as<double>(h->rTallB), m, C, ldc));
    CK(cudaStreamSynchronize(h->ctx.stream));
    CK(cudaGetLastError());
    if (*(volatile int32_t *)(h->h_pin + 1) != 0) {
        g_last_error = "tall product: a bounded device wait gave up";
        return SLRF_ETIMEOUT;
    }
    return SLRF_OK;
}

slrf_status slrf_syev(slrf_handle *h, int32_t m, const double *S, double *lam, double *Q) {
    if (!h || !S || !lam || !Q || m < 1 || m > 1024) return SLRF_EINVAL;
    CKS(ensure(h, h->rSmall, small_syev_work_bytes(m) + (size_t)m * m * sizeof(double)));
    double *Sc = as<double>(h->rSmall);
    double *w = Sc + (size_t)m * m;
    CK(cudaMemcpyAsync(Sc, S, (size_t)m * m * 8, cudaMemcpyDeviceToDevice, h->ctx.stream));
    h->ctx.before(KC_SMALL_DENSE, 16.0 * m * m, 0);
    k_symmetrize<<<(unsigned)(((size_t)m * m + 255) / 256), 256, 0, h->ctx.stream>>>(m, Sc);
    h->ctx.after();
    CK(small_syev(h->ctx, m, Sc, lam, Q, w, h->opts.eig_refine));
    CK(cudaGetLastError());
    return SLRF_OK;
}

slrf_status slrf_rayleigh_ritz(slrf_handle *h, int32_t m, const double *U, int64_t ldu, double *theta, double *X,
                               int64_t ldx, double *resid) {
    if (!h || !theta || !resid || m > 1024) return SLRF_EINVAL;
    CKS(check_dense(U, ldu, m));
    CKS(check_dense(X, ldx, m));
    const int64_t n = h->A.n;
    if (m > n) return SLRF_EINVAL;
    CKS(ensure(h, h->rAX, (size_t)n * m * sizeof(double)));
    CKS(ensure(h, h->rBX, (size_t)n * m * sizeof(double)));
    CKS(ensure(h, h->rRho, (size_t)m * sizeof(double) + (size_t)h->ctx.sm_count * 4 * m * 3 * sizeof(double)));
    int32_t chol[2] = {0, 0};
    CKS(rr_step(h, m, U, ldu, theta, X, ldx, as<double>(h->rAX), as<double>(h->rBX), chol));
    double *rho_ax = as<double>(h->rRho);
    residual(h->ctx, (int)n, m, as<double>(h->rAX), as<double>(h->rBX), m, theta, nullptr, 0, resid, rho_ax,
             rho_ax + m);
    CK(cudaStreamSynchronize(h->ctx.stream));
    CK(cudaGetLastError());
    return (chol[0] || chol[1]) ? SLRF_CHOLQR_FAIL : SLRF_OK;
}

}  // extern "C"
