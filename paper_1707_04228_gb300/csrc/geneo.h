// GenEO coarse space, coarse operators and PCG vector kernels (Section 2.3).
#pragma once

#include "factor.h"

namespace gl {

// Element -> local-index maps of every subdomain (for local products with the
// element matrices): n_pairs entries of (element id, subdomain, 81 local
// indices or -1).
struct LocalElems {
    int64_t n_pairs = 0;
    DBuf<int> elem, sub;
    DBuf<int> loc;   // 81 per pair
};

// y_s += S (K_s) S x_s for every subdomain s: S = diag(xi) if xi != NULL,
// K_s = sum of the subdomain's element matrices (applied matrix-free from C_e
// and the Gauss-point geometry); x, y multi-vectors of nv columns in the
// per-subdomain layout of FactorPlan (x[vec_off*nv + v*n + i]).
void local_K_apply(const FactorPlan &P, const LocalElems &E, const double *C, const double *geo, const double *xi,
                   const double *x, double *y, int nv, cudaStream_t s);

// G_s = A_s^T B_s (k x k per subdomain, row-major k*k block per subdomain), A,
// B multi-vectors of k columns in the FactorPlan layout.
void local_gram(const FactorPlan &P, const double *A, const double *B, int k, double *G, cudaStream_t s);

// Per subdomain: solve G_B y = mu G_M y (k x k, G_M SPD), eigenvectors
// G_M-orthonormal, sorted by mu descending; writes Y (k x k, column a = vector
// a, row-major [b*k + a]) and mu.
void small_geneig(int n_sub, int k, const double *GB, const double *GM, double *Y, double *mu, int *d_err,
                  cudaStream_t s);

// X <- X Y per subdomain (k columns), using tmp of the same size.
void local_rotate(const FactorPlan &P, double *X, const double *Y, int k, double *tmp, cudaStream_t s);

// Deterministic pseudo-random fill of a multi-vector (splitmix64 hash of the index).
void fill_random(double *x, int64_t n, uint64_t seed, cudaStream_t s);

// Coarse operators: Z stored per subdomain as n_s x m column-major (FactorPlan
// layout with nv = m).  c[s*m + a] = sum_i Z_s[i, a] r[gdof_s[i]];
// z[gdof_s[i]] += sum_a Z_s[i, a] y[s*m + a].
void coarse_restrict(const FactorPlan &P, const double *Z, int m, const double *r, double *c, cudaStream_t s);
void coarse_prolong(const FactorPlan &P, const double *Z, int m, const double *y, double *z, cudaStream_t s);

// Scales a multi-vector by xi row-wise: X[:, a] *= xi.
void scale_rows(const FactorPlan &P, double *X, const double *xi, int k, cudaStream_t s);

// ---------------------------------------------------------------- many laminates at once
struct PartDesc {
    int64_t elem_off, dof_off, n_dof;
    int nx, ny, NX, NY;
};
void launch_ku_batch(const PartDesc *d_parts, int n_parts, int64_t n_elem, int64_t n_dof, const double *C,
                     const double *geo, const double *x, double *y, cudaStream_t s);

// Per-part PCG state (structure of arrays, n parts each).
struct SegScalars {
    double *rho, *rho_new, *pq, *rr, *ff, *rz_old;
    int *active, *iters;
};
constexpr int SEG_BLOCKS = 64;
// out[i] = sum over part i's range of a*b   (partials: n * SEG_BLOCKS)
void seg_dot(const double *a, const double *b, const PartDesc *parts, int n, double *partials, double *out,
             cudaStream_t s);
// x += alpha_i p, r -= alpha_i q (alpha_i = rho_i/pq_i for active parts, else 0); rr_i = r.r
void seg_update_xr(double *x, double *r, const double *p, const double *q, const PartDesc *parts, int n,
                   SegScalars S, double *partials, cudaStream_t s);
// p = z + beta_i p, beta_i = (rho_new_i - rz_old_i) / rho_i; then rho_i = rho_new_i
void seg_update_p(double *p, const double *z, const PartDesc *parts, int n, SegScalars S, cudaStream_t s);
// for active parts: iters_i += 1, deactivate when rr_i <= tol^2 ff_i or iters_i >= max_iter; *n_active = count
void seg_check(SegScalars S, int n, double tol, int max_iter, int *n_active, cudaStream_t s);
// with rr_i the FP64 true residual of every part: reactivate the inactive parts that stopped below
// max_iter on a recurrence residual whose true residual misses tol (rr_i > tol^2 ff_i, finite);
// *n_active = how many were reactivated
void seg_confirm(SegScalars S, int n, double tol, int max_iter, int *n_active, cudaStream_t s);

// ---------------------------------------------------------------- PCG vector kernels
struct CGScalars {
    double rho, rho_new, pq, rr, rz_old, alpha, beta, ff;
};

// out = sum a_i b_i (deterministic two-stage reduction) written to *out (device).
void dot(const double *a, const double *b, int64_t n, double *partials, double *out, cudaStream_t s);
// x += alpha p; r -= alpha q, alpha = S->rho / S->pq; partial sums of r.r -> S->rr
void cg_update_xr(double *x, double *r, const double *p, const double *q, int64_t n, CGScalars *S,
                  double *partials, cudaStream_t s);
// beta = rho_new / rho (or flexible), p = z + beta p, rho = rho_new
void cg_update_p(double *p, const double *z, int64_t n, CGScalars *S, cudaStream_t s);
// y[dof[i]] = val (val = 0 or from array)
void set_entries(double *y, const int64_t *dof, int64_t n, const double *vals, cudaStream_t s);
// y = a - b
void sub(double *y, const double *a, const double *b, int64_t n, cudaStream_t s);
void axpy(double *y, double a, const double *x, int64_t n, cudaStream_t s);
void max_where(const double *v, const uint8_t *mask, int64_t n, double *out, cudaStream_t s);

}  // namespace gl
