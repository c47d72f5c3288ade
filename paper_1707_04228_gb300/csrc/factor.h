// Batched multifrontal supernodal Cholesky of many subdomain matrices, and the
// batched triangular solves with the factors (Section 2.3: direct local
// solves of the overlapping Schwarz preconditioner).
#pragma once

#include <mutex>

#include "gl_internal.h"

namespace gl {

// A kernel's dynamic shared-memory limit is an attribute of the device that
// is current when it is set, so the limit already raised is kept per device.
struct SmemLimit {
    static constexpr int MAX_DEVICES = 64;
    std::mutex mu;
    size_t set[MAX_DEVICES] = {};
    template <class F>
    void ensure(size_t need, F apply) {
        int dev = 0;
        GL_CUDA(cudaGetDevice(&dev));
        GL_REQUIRE(dev >= 0 && dev < MAX_DEVICES, "device index out of range");
        std::lock_guard<std::mutex> lock(mu);
        if (need > set[dev]) {
            apply(need);
            set[dev] = need;
        }
    }
};

template <class F>
inline void raise_smem_limit(SmemLimit &L, size_t need, F apply) {
    L.ensure(need, apply);
}

// Per supernode, flattened over all subdomains of one plan.
struct FrontDesc {
    int64_t l_off;      // f x p column-major panel in the factor array
    int64_t row_off;    // f local row indices in the row array
    int64_t front_off;  // front workspace offset (within its level's buffer)
    int64_t vec_off;    // subdomain local-vector offset
    int64_t rel_off;    // q entries: position of each structure row in the parent front
    int64_t pair_off;   // (element, 81 positions) pairs assembling into the front
    int p, q, n_pairs, parent, sub, slot;   // slot: 0/1 = which child of the parent
    int first, vlen;    // first pivot's local index; subdomain local length
};

struct Level {
    std::vector<int> fronts;      // global supernode indices at this depth
    std::vector<int> child_slot[2];
    int max_p = 0, max_f = 0;
    int64_t ws = 0;               // workspace entries used by the level
    DBuf<int> d_fronts, d_child[2];
};

// Per-level timing of the sweeps (gl_profile_levels): while on, every
// factor_solve with one right-hand side records a CUDA event before each
// level's launch and after the last, waits for the last one and adds the
// level times to fwd_ms / bwd_ms (indexed by depth).
struct LevelClock {
    bool on = false;
    std::vector<cudaEvent_t> ev;
    std::vector<double> fwd_ms, bwd_ms;
    int64_t calls = 0;
    LevelClock() = default;
    LevelClock(const LevelClock &) = delete;
    LevelClock &operator=(const LevelClock &) = delete;
    LevelClock(LevelClock &&o) noexcept { swap(o); }
    LevelClock &operator=(LevelClock &&o) noexcept {
        if (this != &o) swap(o);
        return *this;
    }
    ~LevelClock() {
        for (cudaEvent_t e : ev)
            if (e) cudaEventDestroy(e);
    }
    void swap(LevelClock &o) noexcept {
        std::swap(on, o.on);
        ev.swap(o.ev);
        fwd_ms.swap(o.fwd_ms);
        bwd_ms.swap(o.bwd_ms);
        std::swap(calls, o.calls);
    }
};

// Streams and events of the overlapped sweeps (FactorPlan::overlap_top): per
// half of the subdomains a high-priority stream for its top levels and a
// default-priority stream for its deep levels.
struct HalfStreams {
    cudaStream_t hi[2] = {}, lo[2] = {};
    cudaEvent_t fork = nullptr, ev[6] = {};
    HalfStreams() = default;
    HalfStreams(const HalfStreams &) = delete;
    HalfStreams &operator=(const HalfStreams &) = delete;
    ~HalfStreams() {
        for (cudaEvent_t e : ev)
            if (e) cudaEventDestroy(e);
        if (fork) cudaEventDestroy(fork);
        for (int h = 0; h < 2; ++h) {
            if (hi[h]) cudaStreamDestroy(hi[h]);
            if (lo[h]) cudaStreamDestroy(lo[h]);
        }
    }
};

struct FactorPlan {
    int n_sub = 0;
    std::vector<int64_t> vec_off, vec_len;   // per subdomain
    int64_t n_local = 0;                     // total local DOFs
    std::vector<FrontDesc> fr;
    std::vector<Level> levels;               // index = depth
    int64_t l_size = 0;
    int64_t nnz = 0;                         // lower-triangle entries: sum p(p+1)/2 + p q
    int64_t ws_max = 0;
    int max_f = 0;
    double ws_budget_bytes = 6e9;            // numeric_factor: workspace per buffer (subdomain groups fit it)
    bool tc_update = true;                   // FP32 factors: trailing updates on the tensor cores
    bool s20 = false;                        // serendipity elements: element matrices P^T K_Q2 P
    int last_groups = 0;                     // groups the last numeric_factor used
    mutable LevelClock clock;                // per-level sweep timing (off unless profiling)
    // > 0: single right-hand-side sweeps split the subdomains in two halves
    // whose sweeps overlap -- the second half starts when the first reaches
    // its top `overlap_top` levels, and those levels of either half run on a
    // high-priority stream -- so that the deep levels of one half fill the
    // SMs the few large fronts of the other half's top levels leave idle.
    int overlap_top = 0;
    std::vector<int> half_fronts;            // per level: fronts of the first half (a prefix of the list)
    mutable std::unique_ptr<HalfStreams> hs;
    // device
    DBuf<FrontDesc> d_fr;
    DBuf<int> d_rows, d_rel, d_pair_elem;
    DBuf<int16_t> d_pair_pos;
    DBuf<int64_t> d_gdof;                    // local -> global DOF (concatenated)
    DBuf<int64_t> d_vec_off, d_vec_len;      // per subdomain
    std::vector<int64_t> h_gdof;
};

void build_plan(const std::vector<SubSymbolic> &subs, FactorPlan &P, cudaStream_t s);

// Numeric factorisation.  Front entries from the element matrices, formed on
// the fly in FP64 from C_e (36 per element) and the Gauss-point geometry (270
// per element), scaled by (1 + sigma xi_i xi_j) (xi indexed by local DOF, may
// be NULL when sigma == 0).  Factor values of type T, left in the
// partitioned-inverse form that factor_solve reads (every 32-pivot diagonal
// block inverted, the rows below it multiplied by that inverse).
template <class T>
void numeric_factor(FactorPlan &P, const double *C, const double *geo, const double *xi, double sigma, T *L, int *d_err,
                    cudaStream_t s);

// Trailing update of an FP32 level on the tensor cores (syrk_tc.cu): for every
// front with kw = min(syrk_tc_panel(), p - k0) factored panel columns
// [k0, k0 + kw), F[r, c] -= sum_k F[r, k] F[c, k] over base = k0 + kw <= c <= r.
// d_err is set to 2 if a tensor-core wait gave up.
int syrk_tc_panel();
void syrk_tc_level(const int *d_fronts, int n_fronts, const FrontDesc *d_fr, int k0, int max_f, float *ws,
                   int *d_err, cudaStream_t s);

// x <- L^{-T} L^{-1} x (L as factored; stored in partitioned-inverse form)
// for local multi-vectors of kcols columns per subdomain,
// each column of the subdomain's length stored contiguously:
// x[vec_off*kcols + c*n + i] (kcols = 1: plain concatenated local vectors).
template <class T>
void factor_solve(const FactorPlan &P, const T *L, T *x, int kcols, cudaStream_t s);

// Switch the per-level sweep timing on (resetting it) or off.
void level_clock_enable(FactorPlan &P, bool on);

// local <-> global transfers: xl[i] = (T) r[gdof[i]]; z[gdof[i]] += xl[i]
template <class T>
void gather_local(const FactorPlan &P, const double *r, T *xl, cudaStream_t s);
template <class T>
void scatter_add_local(const FactorPlan &P, const T *xl, double *z, cudaStream_t s);

// Block-diagonal y = A x: block b (n_b rows, vector offset voff[b], matrix at aoff[b]).
void dense_symv_blocks(const double *A, const int64_t *aoff, const int *voff, const int *nb, int nblk, int total,
                       const double *x, double *y, cudaStream_t s);
// A^{-1} (n x n, column-major) of a dense SPD A by Cholesky of the front
// [[D A D, I], [I, 0]] (D = diag(A)^{-1/2}; Schur complement -(D A D)^{-1}).
// drop > 0: columns whose pivot on the unit-diagonal scale is <= drop are left
// out (zero rows and columns in Ainv); returns how many were dropped.
int dense_inverse(const double *A, int n, double *Ainv, int *d_err, cudaStream_t s, double drop = 0.0);

}  // namespace gl
