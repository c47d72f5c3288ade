/*
 * geneo_lam.h -- C ABI of the GB300 GenEO-PCG solver for layered laminates.
 *
 * The library solves K u = f (Section 2.3, Eq. eq-1) for 3D anisotropic
 * linear elasticity on a layered, structured hexahedral laminate (Section 2.1,
 * "dune-composites"), discretised with 27-node triquadratic (Q2) hexahedra and
 * full 3x3x3 Gauss integration, by conjugate gradients (Section 2.3) on the
 * preconditioned system P K u = P f (Eq. eq-pre), where P is the two-level
 * overlapping additive Schwarz preconditioner with the GenEO coarse space
 * (Section 2.3, Fig. domaindecomp, Fig. eig).  Stresses sigma_33 = sigma_r and
 * tau_13 = tau_rs (Section 2.2 notation, Eq. eq-Camanho) are recovered at
 * element centres.
 *
 * Conventions (all entry points):
 *   units      N, mm, MPa.
 *   mesh       nx x ny x nz elements, e = ex + nx*(ey + ny*ez); z is the
 *              thickness (r) direction, x the s direction, y the width l.
 *   nodes      (2nx+1)(2ny+1)(2nz+1), n = ix + NX*(iy + NY*iz), x fastest.
 *   DOFs       N = 3 * nodes, dof = 3*n + component (node-major).
 *   faces      0 -s, 1 +s, 2 -l, 3 +l, 4 -r (inner/bottom), 5 +r (outer/top).
 *   pointers   every array argument may be host memory or CUDA device memory
 *              of the context's device; the library tells them apart with
 *              cudaPointerGetAttributes.  Input arrays are caller-owned and
 *              copied before the call returns; output arrays are caller-
 *              allocated with the stated length.  The library allocates and
 *              frees its own device memory; nothing it returns needs freeing
 *              except the context (gl_destroy).
 *   errors     0 on success, a negative GL_ERR_* code otherwise; nothing
 *              throws across the ABI.  gl_last_error() gives a message for the
 *              calling thread's last failure.  A context is not thread-safe;
 *              separate contexts are independent.
 *   streams    all GPU work of a context runs on the stream given to
 *              gl_create (0 = the legacy default stream).  Calls that return
 *              results in host memory synchronise that stream.
 */
#ifndef GENEO_LAM_H
#define GENEO_LAM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    GL_OK = 0,
    GL_ERR_INVALID_ARG = -1,
    GL_ERR_OOM = -2,
    GL_ERR_CUDA = -3,
    GL_ERR_NOT_SPD = -4,        /* a Cholesky pivot was <= 0 (local or coarse factor) */
    GL_ERR_NOT_CONVERGED = -5,  /* max_iter reached; info and u still filled */
    GL_ERR_NAN = -6,            /* a NaN or Inf appeared in the iteration */
    GL_ERR_TIMEOUT = -7,        /* a device-side wait gave up (e.g. on the tensor cores) */
    GL_ERR_STATE = -8           /* call out of order (e.g. solve before setup) */
};

enum { GL_PREC_FP64 = 0, GL_PREC_MIXED = 1 };

typedef struct gl_ctx gl_ctx;

/* Orthotropic ply constants (Table 1, Section 2.2).  nu_ij = -eps_j/eps_i
 * under uniaxial stress along i.  MPa. */
typedef struct {
    double E1, E2, E3, G12, G13, G23, nu12, nu13, nu23;
} gl_ortho;

/* Layered structured mesh (Section 2.2 stacking sequences; Section 3 curved
 * map x = L + r sin(psi), y = l, z = r cos(psi), psi = arc * t on the arc).
 *   x[nx+1]  s vertex coordinates: mm for geometry 0 (flat); for geometry 1
 *            (curved) a parametric t: limb 1 on [-1,0], the arc on [0,1],
 *            limb 2 on [1,2] (limbs of length limb_L appended tangentially).
 *   y[ny+1]  width vertex coordinates, mm.
 *   layers   nlayers layers from the inner (r = R_inner, or z = 0) face out:
 *            layer_nel[k] elements of equal thickness layer_thick[k]/nel;
 *            layer_mat[k] indexes the material table (orthotropic entries
 *            first, then isotropic); layer_angle_deg[k] is the ply angle about
 *            the laminate normal.
 *   theta_e  per-element fibre misalignment angle (rad, rotation about the
 *            width axis l), length nx*ny*nz, or NULL for zero.
 *   node_dr  per-node offset (mm) added to the through-thickness coordinate
 *            (depth r from the inner face, or z when flat) before the curved
 *            map: a geometric wrinkle r^ = r + f(s, l, r) as in Section 3
 *            (Eq. eq-wrinkle); length (2nx+1)(2ny+1)(2nz+1) in node order (x
 *            fastest, then y, then z), or NULL.  The offset nodes must keep
 *            every through-thickness node column strictly increasing, else
 *            gl_set_mesh returns GL_ERR_INVALID_ARG.
 *   elem_mat per-element material index (into the same table as layer_mat)
 *            overriding the element's layer, length nx*ny*nz, or NULL: e.g.
 *            resin strips along the free edges of the width (Section 3).
 *   element  0: 27-node triquadratic Q2 hexahedra; 1: the 20-node serendipity
 *            hexahedra of Section 2.1 (the paper's element: vertices and edge
 *            midpoints, full 3x3x3 Gauss integration).  The serendipity mesh
 *            keeps the Q2 node numbering: its nodes are the grid nodes with at
 *            most one odd index, and the other (face- and body-centre) entries
 *            of every N-vector are not unknowns -- the solver eliminates them,
 *            gl_solve and gl_solve_increment return there the values of the
 *            serendipity field (so the vector is also its Q2 representation),
 *            and the other calls ignore what they hold on input, except
 *            gl_stress_noalloc, which reads u as given.  Not available in
 *            gl_batch_*.
 *   periodic_width  1: periodic conditions across the width (Section 3, the
 *            39-ply study), u(s, l = y[0], r) = u(s, l = y[ny], r): every node
 *            of the last width plane is identified with its partner on the
 *            first.  The last plane's entries of N-vectors are handled like
 *            the serendipity centres above (not unknowns; returned equal to
 *            the first plane's).  Needs py = 1 (every subdomain spans the
 *            width), ny >= 2 and element 0; not available in gl_batch_*.
 *            Tractions on the faces l = y[0], y[ny] do not apply.
 * Material axes: R = R_l(psi + theta_e) R_r(phi), psi the frame angle at the
 * element centre (0 on limb 1 and flat plates), C_e constant per element. */
typedef struct {
    int nx, ny;
    const double *x, *y;
    int nlayers;
    const int *layer_nel;
    const double *layer_thick;
    const int *layer_mat;
    const double *layer_angle_deg;
    int geometry;              /* 0 flat, 1 curved */
    double R_inner, limb_L, arc_deg;
    const double *theta_e;
    const double *node_dr;
    const int *elem_mat;
    int element;               /* 0 Q2, 1 serendipity-20 */
    int periodic_width;        /* 0 or 1 */
} gl_mesh;

/* Solver options.
 *   px,py,pz   subdomains per axis (element boxes of near-equal size, the
 *              first n % p boxes one element larger), grown by `overlap`
 *              element layers (>= 1) (Section 2.3, Fig. domaindecomp).
 *   nev        GenEO eigenvectors kept per subdomain (0 = one-level Schwarz).
 *   max_iter   PCG iteration cap.
 *   precision  GL_PREC_FP64, or GL_PREC_MIXED (FP32 local factors and solves
 *              inside FP64 CG, FP64 coarse solve, flexible beta, residual
 *              replacement every resid_period iterations).
 *   tol        stop when ||r_k||_2 / ||r_0||_2 <= tol, r_0 = f (x_0 = 0).
 *   sigma      shift of the definite GenEO pencil (eigenvectors do not
 *              depend on it); <= 0 selects 1e-3.
 *   eig_iters  cap on the subspace iterations of the GenEO eigensolver
 *              (<= 0: 100); after at least 4 iterations it stops once the
 *              kept Ritz values of every subdomain change by less than 1e-10
 *              (relative) between iterations.
 *   factor_ws_bytes  device workspace per buffer of the numeric
 *              factorisation (two buffers hold the dense fronts of two
 *              adjacent dissection levels); subdomains are factored in
 *              consecutive groups that fit it.  <= 0 selects 6e9.  A smaller
 *              value only adds groups (more launches), never changes results.
 *   eig_group_bytes  device memory for the shifted Neumann factors of one
 *              group of subdomains in the GenEO eigensolver; the subdomains
 *              are processed in consecutive groups that fit it.  <= 0 selects
 *              4e10.  The random start vectors of the subspace iteration are
 *              drawn per group, so another grouping changes the eigenvectors
 *              within the eigensolver's convergence, not the solution of a
 *              converged solve beyond its tolerance.
 *   fp32_update  GL_PREC_MIXED only: how the FP32 local factorisation updates
 *              its trailing matrices.  0 (default): 128-column panels whose
 *              rank-128 trailing updates run on the tensor cores (tcgen05,
 *              TF32 inputs split hi + lo, FP32 accumulation: FP32-level
 *              accuracy); 1: rank-32 updates on the FP32 CUDA cores.
 *   sweep_overlap  how the triangular solves of the PCG iteration are
 *              scheduled.  The subdomains are split in two halves whose
 *              sweeps overlap: the second half starts when the first reaches
 *              its top sweep_overlap dissection levels, and those levels of
 *              either half run on a high-priority stream, so that one half's
 *              many small deep fronts fill the SMs that the other half's few
 *              large top fronts leave idle.  0 selects the default, every
 *              level counted as top (the halves sweep concurrently, both at
 *              high priority); < 0 sweeps sequentially.  Same arithmetic
 *              either way.  Single laminates (gl_setup) only; timed phases
 *              (gl_profile) sweep sequentially. */
typedef struct {
    int px, py, pz, overlap, nev, max_iter, precision, resid_period;
    double tol, sigma;
    int eig_iters;
    double factor_ws_bytes, eig_group_bytes;
    int fp32_update;
    int sweep_overlap;
} gl_opts;

/* Results of one solve.  rel_resid_true = ||f - K u||_2 / ||f||_2 on the
 * free DOFs, recomputed in FP64 after the iteration. */
typedef struct {
    int iters;
    int status;
    double rel_resid;        /* last recurrence residual ratio */
    double rel_resid_true;
    double ms_setup, ms_solve;
    int64_t n_free;
    int n_coarse;            /* coarse-space dimension sum_j m_j */
    int64_t factor_nnz;      /* stored entries of all local factors */
    int n_coarse_dropped;    /* coarse columns left out of K_0's Cholesky as
                                linearly dependent (pivot <= 1e-10 with K_0
                                scaled to unit diagonal), e.g. two subdomains
                                that coincide on a narrow laminate */
} gl_info;

/* Context on CUDA device `device`; `cuda_stream` is a cudaStream_t (or NULL). */
int gl_create(gl_ctx **out, int device, void *cuda_stream);
void gl_destroy(gl_ctx *ctx);
const char *gl_strerror(int code);
const char *gl_last_error(void);

/* Material table: n_ortho orthotropic entries, then n_iso isotropic (E, nu)
 * pairs (Table 1, Section 2.2). */
int gl_set_materials(gl_ctx *ctx, int n_ortho, const gl_ortho *ortho, int n_iso,
                     const double *E_nu_pairs);
int gl_set_mesh(gl_ctx *ctx, const gl_mesh *mesh);
/* Prescribed displacements: n DOF indices (int64) and values (mm). */
int gl_set_dirichlet(gl_ctx *ctx, int64_t n, const int64_t *dof, const double *val);
/* Uniform surface traction t[3] (MPa, global axes) on one box face; repeated
 * calls add up.  Consistent nodal loads by 3x3 face Gauss quadrature. */
int gl_set_traction(gl_ctx *ctx, int face, const double t[3]);

/* Builds geometry, element stiffness data, the decomposition, the local
 * nested-dissection supernodal Cholesky factors, the GenEO coarse space and
 * the coarse Cholesky factor (Section 2.3). */
int gl_setup(gl_ctx *ctx, const gl_opts *opts);

int gl_num_dofs(const gl_ctx *ctx, int64_t *n_dof);
int gl_num_elems(const gl_ctx *ctx, int64_t *n_elem);
/* Assembled load vector f (length N) of the tractions. */
int gl_rhs(gl_ctx *ctx, double *f);

/* PCG solve of K u = f with the prescribed Dirichlet values.  f has length N
 * (NULL = the assembled tractions); entries at Dirichlet DOFs are ignored.
 * u (length N, out) holds the full displacement, prescribed values included.
 * info may be NULL. */
int gl_solve(gl_ctx *ctx, const double *f, double *u, gl_info *info);

/* Increment of a solution whose prescribed values are already in place: PCG
 * solve of K_ff du_f = g_f with du = 0 on the Dirichlet DOFs (g of length N,
 * required; its Dirichlet entries are ignored), stopping when
 * ||g_f - K_ff du_f|| <= tol ||g_f||.  For a change of the stiffness K -> K',
 * u' = u + du with g = f - K' u solves the new problem; with the residual of
 * u left out, g = -(K' - K) u, du is the change of u to first order in the
 * solver tolerance of du alone (used for finite differences with respect to
 * theta_e, where only element e contributes to g). */
int gl_solve_increment(gl_ctx *ctx, const double *g, double *du, gl_info *info);

/* Stress recovery at element centres (Section 2.2 notation): s33 = sigma_rr,
 * t13 = tau_rs in the local (s, l, r) frame, length nx*ny*nz each (either may
 * be NULL); peak_s33 (may be NULL) = the maximum of s33 over the isotropic
 * resin-interface elements. */
int gl_stress(gl_ctx *ctx, const double *u, double *s33, double *t13, double *peak_s33);

/* Stress recovery that allocates nothing.  The paper has no counterpart: this
 * entry point is for callers that cannot allocate device memory while they
 * run -- a host framework that has handed nearly all device memory to its own
 * caching pool (the local factors leave little free), a latency-bound loop in
 * which cudaMalloc or cudaFree would synchronise the device and stall the
 * other streams, or a deployment whose device footprint must stay fixed once
 * the library is loaded.  It computes what gl_stress computes, with these
 * differences:
 *   - u (N entries), s33 and t13 (n_elem each) and peak_s33 (one double, may
 *     be NULL) must be device memory of the context's device, allocated by
 *     the caller; anything else, and a buffer whose device allocation ends
 *     before the entries the call touches (checked with cuMemGetAddressRange:
 *     a short view into a larger allocation is not caught), is rejected with
 *     GL_ERR_INVALID_ARG before any work is queued;
 *   - it calls no cudaMalloc, cudaFree or allocating library routine: the
 *     partial maxima of the resin peak live in a fixed array of 16,384
 *     doubles (128 KB) inside the library, which every GPU that loads the
 *     library holds until the process exits; meshes of more than 4,194,304
 *     elements are rejected with GL_ERR_INVALID_ARG;
 *   - the work is queued on the context's stream and the call returns without
 *     waiting for it;
 *   - the first call on a device looks up the array's device address and
 *     caches it.  With lazy module loading (the CUDA default) that first call
 *     is also when the driver loads the library's module, and with it the
 *     128 KB array, onto that device; make the first call before any stream
 *     capture begins and before the caller's device memory is committed;
 *     later calls allocate nothing;
 *   - all calls on a device share the one array, which keeps the last call's
 *     contents.  Each call writes every slot it reads before reading it, so
 *     nothing has to be cleared between calls, but calls whose work overlaps
 *     on the GPU (other streams, other contexts) race on it: order them on
 *     one stream or synchronise between them. */
int gl_stress_noalloc(gl_ctx *ctx, const double *u, double *s33, double *t13, double *peak_s33);

/* Quadratic damage-onset criterion (Section 3.2, Eq. eq-Camanho), per element:
 *   F = sqrt((max(sigma_r, 0)/s33)^2 + (tau_rs/s13)^2 + (tau_rl/s13)^2)
 * from the element-centre stresses in the local (s, l, r) frame, applied in
 * the isotropic resin interfaces only (F = 0 elsewhere).  The paper's
 * allowables are s33 = 61 MPa and s13 = 97 MPa.  F (n_elem, may be NULL);
 * peak (may be NULL) = the largest F; peak_elem (may be NULL) = its element
 * (ties within about 1e-5 relative may resolve to either element).  At most
 * 16,777,215 elements. */
int gl_failure_index(gl_ctx *ctx, const double *u, double s33_allow, double s13_allow, double *F, double *peak,
                     int64_t *peak_elem);

/* Gradients with respect to the per-element misalignment angles theta_e
 * (adjoint method; the objective is any function of the centre stresses).
 *
 * gl_set_theta: replaces theta_e (length nx*ny*nz, rad).  After gl_setup the
 *   element stiffness tensors C_e are recomputed at once; the local factors
 *   and the coarse space built for the previous angles are kept and still
 *   serve as the (SPD) preconditioner, so later solves use K(theta_new).
 * gl_stress_vjp: vector-Jacobian product of gl_stress at displacement u (N):
 *   dJdu (N, may be NULL) = sum_e (w33_e d s33_e/du + w13_e d t13_e/du) and
 *   dJdtheta (n_elem, may be NULL) = sum of the same weights times the partial
 *   derivatives of s33_e, t13_e with respect to theta_e at fixed u.  w33, w13
 *   (n_elem) may be NULL (zero).
 * gl_adjoint: solves K_ff lambda = (dJdu)_f (lambda = 0 on Dirichlet DOFs) by
 *   PCG with the setup's preconditioner, then writes
 *   grad[e] = -lambda_e^T (dK_e/dtheta_e) u_e for every element (n_elem),
 *   dK_e/dtheta_e = sum_q w_q |J_q| B_q^T (dC_e/dtheta_e) B_q.  The total
 *   derivative of J is grad + dJdtheta from gl_stress_vjp.  info (may be NULL)
 *   describes the adjoint solve. */
int gl_set_theta(gl_ctx *ctx, const double *theta_e);
int gl_stress_vjp(gl_ctx *ctx, const double *u, const double *w33, const double *w13, double *dJdu,
                  double *dJdtheta);
int gl_adjoint(gl_ctx *ctx, const double *u, const double *dJdu, double *grad, gl_info *info);

/* Operator pieces, for parity checks against an assembled reference.
 * gl_apply_K: y = K x over all N DOFs (no Dirichlet elimination), the
 *   matrix-free element-by-element product of Eq. eq-1.
 * gl_apply_prec: z = M^{-1} r with M^{-1} = Z K_0^{-1} Z^T + sum_j R_j^T
 *   A_j^{-1} R_j (Section 2.3); r, z of length N, Dirichlet entries ignored
 *   on input and zero on output.
 * gl_geneo_eigenvalues: the kept GenEO eigenvalues, subdomain-major
 *   (n_sub * nev entries; lambda ascending within a subdomain). */
int gl_apply_K(gl_ctx *ctx, const double *x, double *y);
int gl_apply_prec(gl_ctx *ctx, const double *r, double *z);
int gl_geneo_eigenvalues(gl_ctx *ctx, double *lambda, int capacity, int *count);

/* Many laminates solved together (the batched form of the method: every
 * laminate keeps its own decomposition, local factors, GenEO coarse space
 * and PCG scalars; their vectors are concatenated so that each phase of the
 * iteration -- K u, the local forward/backward sweeps of all subdomains of
 * all laminates, the coarse step, the per-laminate reductions -- is one
 * launch, and one PCG iteration of the whole batch is replayed as a CUDA
 * graph).  Laminates that converge stop updating; the others go on.
 *
 * gl_batch_create: n contexts with materials, mesh, Dirichlet data and
 *   tractions set (no gl_setup needed); they must live on one device and
 *   stay alive while the batch exists; their stream is replaced by the
 *   batch's until gl_batch_destroy gives each its own back.  cuda_stream may be NULL (the batch creates a non-blocking
 *   stream; graph capture cannot use the legacy default stream).
 * gl_batch_setup: opts as for gl_setup except px, py: <= 0 selects, per
 *   laminate, the in-plane subdomain grid (px, py, 1) with 8 <= px py <= 64
 *   that minimises a cost model of one solve (setup flops and per-iteration
 *   bytes/flops from the symbolic factorisation of a representative
 *   subdomain); pz is ignored (subdomains span the thickness).
 * gl_batch_solve: u[i] (length N_i, host or device) receives laminate i's
 *   displacement; infos (n entries, may be NULL) its iteration count,
 *   status and residuals.  Returns the worst status.
 * gl_batch_grid: the (px, py) chosen for every laminate (2n ints). */
typedef struct gl_batch gl_batch;
int gl_batch_create(gl_batch **out, int n, gl_ctx *const *items, void *cuda_stream);
int gl_batch_setup(gl_batch *batch, const gl_opts *opts);
int gl_batch_solve(gl_batch *batch, double *const *u, gl_info *infos);
int gl_batch_grid(const gl_batch *batch, int *pxpy);
void gl_batch_destroy(gl_batch *batch);

/* Measurement.  gl_profile(ctx, 1) switches on CUDA-event timing of the
 * solve's phases on the context's stream (matrix-free K u; local Schwarz
 * solves = gather + forward/backward sweeps over all factor levels + scatter,
 * in their normal schedule; coarse restrict/solve/prolong, which then runs
 * after the local solves instead of beside them) and resets the
 * accumulators; gl_profile(ctx, 2) also times every dissection level
 * (gl_profile_levels), the levels then running one after another; 0
 * switches timing off; other values are GL_ERR_INVALID_ARG.  Timing adds a
 * host wait before each phase is reused.
 * gl_profile_read returns the accumulators and the sizes that turn them into
 * bandwidth and flop rates.  gl_kernel_launches returns the number of kernels
 * this library has launched from gl_solve and the gl_apply_* calls since it
 * was loaded (process-wide). */
typedef struct {
    double ms_ku, ms_local, ms_coarse;
    int64_t n_ku, n_local, n_coarse;     /* timed calls of each phase */
    int64_t factor_entries;              /* stored entries of all local factor panels */
    int64_t local_dofs;                  /* sum of the subdomain sizes */
    int factor_bytes_per_entry;          /* 8 (FP64) or 4 (mixed) */
    int factor_levels;                   /* non-empty dissection levels (2 sweeps each) */
    int64_t n_elem, n_dof;
    int n_sub, n_coarse_dim;
    int64_t factor_nonzeros;             /* entries of the lower-triangular factors
                                            (sum over fronts of p(p+1)/2 + p q):
                                            what the two sweeps read and multiply */
    int factor_groups;                   /* subdomain groups of the local factorisation */
    int eig_groups;                      /* subdomain groups of the GenEO eigensolver */
    int max_level_fronts;                /* fronts of the most populated dissection level */
} gl_profile_data;
int gl_profile(gl_ctx *ctx, int enable);
int gl_profile_read(gl_ctx *ctx, gl_profile_data *out);
/* Per dissection level of the local solves (Section 2.3), from the
 * preconditioner applications timed since gl_profile(ctx, 2) (CUDA events
 * before every level's launch; each timed application waits for its last
 * launch).  For every depth d < min(max_levels, *n_levels): fwd_ms[d] and
 * bwd_ms[d], the summed milliseconds of that level's forward and backward
 * sweep launches; fronts[d], its fronts over all subdomains; nonzeros[d],
 * their factor entries (sum of p(p+1)/2 + p q, what each sweep reads and
 * multiplies once); padded[d], the entries of the 32-column block panels
 * the kernels multiply (sum over blocks of 32 x the rows from the block
 * down: the diagonal blocks' upper triangles and the last block's missing
 * columns count as zeros); max_front[d], the rows of its largest front.
 * *n_levels = number of levels, *calls = timed
 * applications.  Every output pointer is host memory and may be NULL.
 * Errors: GL_ERR_STATE before gl_setup, GL_ERR_INVALID_ARG for
 * max_levels < 0. */
int gl_profile_levels(gl_ctx *ctx, int max_levels, double *fwd_ms, double *bwd_ms, int64_t *fronts,
                      int64_t *nonzeros, int64_t *padded, int *max_front, int *n_levels, int64_t *calls);
long long gl_kernel_launches(void);

/* FP64 FMA throughput of device `device`, measured: every thread of 8 blocks
 * of 256 per SM runs 8 independent chains of `iters` dependent FP64 FMAs
 * (no memory traffic), `reps` timed launches after one warm-up, CUDA events
 * on a stream of its own.  flops_per_s = 2 x FMAs / time; n_sm (may be NULL)
 * = the device's multiprocessor count; ms (may be NULL) = the timed span.
 * This is the peak against which the FP64-bound kernels (K u, FP64 local
 * sweeps) report their fraction. */
int gl_fp64_peak_probe(int device, int iters, int reps, double *flops_per_s, int *n_sm, double *ms);

#ifdef __cplusplus
}
#endif
#endif /* GENEO_LAM_H */
