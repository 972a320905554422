// Smoothed-aggregation multigrid hierarchy of a pencil (A, B) (host side).
//
// The shifted systems (A - sigma_j B) y = f of Section 1, Eq. (2) have poles
// with a large imaginary part (Section 3.1: sigma = gamma x (1 + i alpha)),
// the setting in which a multigrid cycle with Jacobi smoothing is an
// effective preconditioner for a shifted Laplace-type operator.  One
// hierarchy serves every pole: the prolongators P_l are built from A alone
// and the Galerkin coarse pencils (P^T A P, P^T B P) keep the pair form, so
// the coarse operator of pole j is A_c - sigma_j B_c on every level.  The
// coarsest pencil is diagonalised once, V^T A_c V = diag(lambda),
// V^T B_c V = I, which gives its exact shifted inverse for any pole:
// (A_c - sigma B_c)^{-1} = V (diag(lambda) - sigma)^{-1} V^T.
#pragma once
#include <stdint.h>

#include <string>
#include <vector>

namespace slrf {

struct HostCsr {
    int n_rows = 0, n_cols = 0;
    std::vector<int32_t> ptr, col;
    std::vector<double> val;
};

struct HostLevel {
    int n = 0;                          // rows of this level
    // pencil of this level (union pattern, pair values); empty for level 0,
    // which is the caller's pencil
    std::vector<int32_t> ptr, col;
    std::vector<double> a, b;
    std::vector<double> diag_a, diag_b;
    double rho = 1.0;                   // spectral radius of D^{-1} A (levels that are smoothed)
    double maxba = 0.0;                 // max_i b_ii / a_ii: |sigma| maxba is the shift's weight on the diagonal
    // transfer to the next level (empty on the coarsest level)
    HostCsr P;    // n x n_next
    HostCsr Rt;   // n_next x n, the transpose of P
    // level 0 only (when it has a next level): the products A P and B P on
    // their common pattern (rows sorted by column) with P's values on that
    // pattern (zero where P has no entry; supp P is inside it since a_ii > 0).
    // The device folds them into the pair matrix (M - D^{-1}) P of the fused
    // finest-level restriction and prolongation.
    std::vector<int32_t> fptr, fcol;
    std::vector<double> fp, fap, fbp;
    // levels >= 1 of a hierarchy built from a near-null space: this level's
    // near-null space (n x n_null, row-major; the stacked R factors), with
    // n_null dofs per node
    std::vector<double> nullspace;
    int n_null = 0;
};

struct MgParams {
    int block = 1;           // dofs per node (1, or 3 for 3-dof elasticity)
    int coarse_target = 256; // stop coarsening at or below this size
    int max_levels = 10;
    double theta = 0.08;     // strength-of-connection threshold
    bool defer_coarse_eig = false;   // leave V, lam to mg_coarse_eig (run concurrently)
    // Optional near-null space of A on level 0: n x n_null, row-major (for
    // 3-dof elasticity the six rigid-body modes, with block = 3).  Without it
    // each aggregate's tentative prolongator block is the constant per dof
    // component; with it, the orthonormal factor Q of the thin QR of the
    // aggregate's rows of the near-null space (aggregates smaller than
    // n_null / block nodes are first merged into a neighbour, and a rank
    // deficient block is completed with unit vectors), and the R factors form
    // the next level's near-null space, with n_null dofs per coarse node.
    const double *near_null = nullptr;
    int n_null = 0;
};

struct HostHierarchy {
    std::vector<HostLevel> lv;   // lv[0] .. lv[nlev-1]; the last is the coarsest
    std::vector<double> V;       // coarsest: n_c x n_c row-major, B_c-orthonormal eigenvectors
    std::vector<double> lam;     // coarsest: eigenvalues, ascending
    double ms_setup = 0.0;
};

// The finest level's pair matrix F = (M - D^{-1}) P in the two layouts of the
// fused restriction (coarse rows of F^T: "down") and prolongation (groups of R
// fine rows with the union of their coarse columns, R pairs per entry: "up"),
// unfolded: per stored pair q holds (A P, B P, a_ii P, b_ii P), and for a
// damping D = (omega / rho_0) / (a_ii - sigma b_ii),
// F = (q0 - kappa q2) - sigma (q1 - kappa q3), kappa = rho_0 / omega.
struct FusedLayout {
    int R = 1;
    std::vector<int32_t> up_ptr, up_col;       // ceil(n / R) + 1 groups; coarse columns
    std::vector<int32_t> down_ptr, down_col;   // n_c + 1 coarse rows; fine columns
    std::vector<int32_t> down_src;             // per down entry: its position in A P's pattern
    // doubles of the values: 4 per stored pair, up pairs (R per entry), then down
    size_t q_count() const { return (up_col.size() * (size_t)R + down_col.size()) * 4; }
};
// From level 0 of a hierarchy with at least two levels (L0.fptr non-empty):
// the two patterns, then the values written to q (q_count() doubles).
void mg_fused_pattern(const HostLevel &L0, int n_coarse, int R, FusedLayout &out);
void mg_fused_values(const HostLevel &L0, const FusedLayout &FL, double *q);

// Build the hierarchy of the n x n pencil given in CSR with shared pattern
// (a = A values, b = B values).  Returns an empty string on success, else a
// description of the failure (non-positive diagonal, coarse mass matrix not
// positive definite, coarsening stalled).
std::string mg_build(int n, const int32_t *ptr, const int32_t *col, const double *a, const double *b,
                     const MgParams &prm, HostHierarchy &H);

// V^T A_l V = diag(lam), V^T B_l V = I for a level with a pencil copy (n_l x n_l
// row-major V, lam ascending); used for the coarsest level and, on demand, for
// the level at which a deep shift truncates the cycle.
std::string mg_level_eig(const HostLevel &L, std::vector<double> &V, std::vector<double> &lam);

// The coarsest level's V, lam of a hierarchy built with defer_coarse_eig
// (and the release of a single level's pencil copy).
std::string mg_coarse_eig(HostHierarchy &H);

// Dense symmetric eigensolver (FP64, host): S = Q diag(w) Q^T, w ascending,
// Q row-major n x n with the eigenvectors in its columns.  S is overwritten.
void host_syev(int n, std::vector<double> &S, std::vector<double> &w, std::vector<double> &Q);

}  // namespace slrf
