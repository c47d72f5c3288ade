// GenEO coarse-space kernels, coarse restrict/prolong, PCG vector kernels.
//
// Section 2.3 (Fig. eig): on each subdomain a few of the lowest-energy modes
// of a local generalised eigenproblem are computed and glued with a
// partition of unity into the coarse space.  The eigenproblem solved here is
// A_j^N p = lambda B_j p with B_j = Xi_j A_j^N Xi_j, through the definite
// pencil B p = mu (A^N + sigma B) p (largest mu <-> smallest lambda), by block
// subspace iteration with Rayleigh-Ritz; these are its batched pieces.
#include <algorithm>

#include "geneo.h"

namespace gl {

constexpr int NV_MAX = 32;

// (local element products: local_K_apply in ku.cu, matrix-free)

// ---------------------------------------------------------------- Gram matrices

constexpr int GRAM_ROWS = 64;

__global__ void __launch_bounds__(256) k_gram(const int64_t *__restrict__ voff, const int64_t *__restrict__ vlen,
                                              const double *__restrict__ A, const double *__restrict__ B, int k,
                                              double *__restrict__ G) {
    const int s = blockIdx.x;
    const int64_t n = vlen[s], base = voff[s] * k;
    const int64_t r0 = (int64_t)blockIdx.y * GRAM_ROWS;
    if (r0 >= n) return;
    const int rows = (n - r0) < GRAM_ROWS ? (int)(n - r0) : GRAM_ROWS;
    __shared__ double sa[NV_MAX][GRAM_ROWS], sb[NV_MAX][GRAM_ROWS];
    for (int idx = threadIdx.x; idx < k * GRAM_ROWS; idx += blockDim.x) {
        int i = idx % GRAM_ROWS, a = idx / GRAM_ROWS;
        bool ok = i < rows;
        sa[a][i] = ok ? A[base + a * n + r0 + i] : 0.0;
        sb[a][i] = ok ? B[base + a * n + r0 + i] : 0.0;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < k * k; idx += blockDim.x) {
        int a = idx / k, b = idx % k;
        double acc = 0.0;
        for (int i = 0; i < rows; ++i) acc += sa[a][i] * sb[b][i];
        atomicAdd(G + (int64_t)s * k * k + idx, acc);
    }
}

void local_gram(const FactorPlan &P, const double *A, const double *B, int k, double *G, cudaStream_t s) {
    if (k > NV_MAX) fail(GL_ERR_INVALID_ARG, "local_gram: too many vectors");
    int64_t maxn = 0;
    for (auto v : P.vec_len) maxn = std::max(maxn, v);
    GL_CUDA(cudaMemsetAsync(G, 0, sizeof(double) * P.n_sub * k * k, s));
    dim3 g(P.n_sub, (unsigned)((maxn + GRAM_ROWS - 1) / GRAM_ROWS));
    k_gram<<<g, 256, 0, s>>>(P.d_vec_off.p, P.d_vec_len.p, A, B, k, G);
    GL_CUDA(cudaGetLastError());
}

// ---------------------------------------------------------------- small generalised eigenproblems

// One thread per subdomain: Cholesky G_M = L L^T, C = L^{-1} G_B L^{-T},
// cyclic Jacobi on C, Y = L^{-T} Q, sort by eigenvalue descending.
__global__ void k_small_geneig(int n_sub, int k, const double *__restrict__ GB, const double *__restrict__ GM,
                               double *__restrict__ Y, double *__restrict__ mu, int *__restrict__ err,
                               double *__restrict__ work) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_sub) return;
    const int kk = k * k;
    double *Lm = work + (int64_t)s * 3 * kk, *C = Lm + kk, *Q = C + kk;
    for (int i = 0; i < kk; ++i) {
        Lm[i] = GM[(int64_t)s * kk + i];
        C[i] = GB[(int64_t)s * kk + i];
    }
    // symmetrise
    for (int i = 0; i < k; ++i)
        for (int j = 0; j < i; ++j) {
            double a = 0.5 * (Lm[i * k + j] + Lm[j * k + i]);
            Lm[i * k + j] = Lm[j * k + i] = a;
            double b = 0.5 * (C[i * k + j] + C[j * k + i]);
            C[i * k + j] = C[j * k + i] = b;
        }
    // Cholesky (lower, row-major L[i*k+j], j <= i)
    for (int j = 0; j < k; ++j) {
        double d = Lm[j * k + j];
        for (int t = 0; t < j; ++t) d -= Lm[j * k + t] * Lm[j * k + t];
        if (!(d > 0.0)) {
            atomicExch(err, 1);
            d = 1e-300;
        }
        d = sqrt(d);
        Lm[j * k + j] = d;
        for (int i = j + 1; i < k; ++i) {
            double v = Lm[i * k + j];
            for (int t = 0; t < j; ++t) v -= Lm[i * k + t] * Lm[j * k + t];
            Lm[i * k + j] = v / d;
        }
    }
    // C <- L^{-1} C (columns), then C <- (L^{-1} C^T): C = L^{-1} G_B L^{-T}
    for (int pass = 0; pass < 2; ++pass) {
        for (int c = 0; c < k; ++c)
            for (int i = 0; i < k; ++i) {
                double v = C[i * k + c];
                for (int t = 0; t < i; ++t) v -= Lm[i * k + t] * C[t * k + c];
                C[i * k + c] = v / Lm[i * k + i];
            }
        for (int i = 0; i < k; ++i)
            for (int j = 0; j < i; ++j) {
                double a = C[i * k + j];
                C[i * k + j] = C[j * k + i];
                C[j * k + i] = a;
            }
    }
    for (int i = 0; i < kk; ++i) Q[i] = 0.0;
    for (int i = 0; i < k; ++i) Q[i * k + i] = 1.0;
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int i = 0; i < k; ++i)
            for (int j = 0; j < k; ++j) {
                double v = C[i * k + j] * C[i * k + j];
                tot += v;
                if (i != j) off += v;
            }
        if (off <= 1e-30 * tot) break;
        for (int p = 0; p < k - 1; ++p)
            for (int q = p + 1; q < k; ++q) {
                double apq = C[p * k + q];
                if (fabs(apq) < 1e-300) continue;
                double app = C[p * k + p], aqq = C[q * k + q];
                double tau = (aqq - app) / (2.0 * apq);
                double t = (tau >= 0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                double c = 1.0 / sqrt(1.0 + t * t), sn = t * c;
                for (int r = 0; r < k; ++r) {   // columns p, q
                    double a = C[r * k + p], b = C[r * k + q];
                    C[r * k + p] = c * a - sn * b;
                    C[r * k + q] = sn * a + c * b;
                }
                for (int r = 0; r < k; ++r) {   // rows p, q
                    double a = C[p * k + r], b = C[q * k + r];
                    C[p * k + r] = c * a - sn * b;
                    C[q * k + r] = sn * a + c * b;
                }
                for (int r = 0; r < k; ++r) {
                    double a = Q[r * k + p], b = Q[r * k + q];
                    Q[r * k + p] = c * a - sn * b;
                    Q[r * k + q] = sn * a + c * b;
                }
            }
    }
    // Y = L^{-T} Q (back substitution per column), order by eigenvalue descending
    int order[NV_MAX];
    for (int i = 0; i < k; ++i) order[i] = i;
    for (int i = 1; i < k; ++i) {
        int v = order[i], j = i - 1;
        while (j >= 0 && C[order[j] * k + order[j]] < C[v * k + v]) {
            order[j + 1] = order[j];
            --j;
        }
        order[j + 1] = v;
    }
    for (int a = 0; a < k; ++a) {
        int src = order[a];
        mu[(int64_t)s * k + a] = C[src * k + src];
        double col[NV_MAX];
        for (int i = k - 1; i >= 0; --i) {
            double v = Q[i * k + src];
            for (int t = i + 1; t < k; ++t) v -= Lm[t * k + i] * col[t];
            col[i] = v / Lm[i * k + i];
        }
        for (int b = 0; b < k; ++b) Y[(int64_t)s * kk + b * k + a] = col[b];
    }
}

void small_geneig(int n_sub, int k, const double *GB, const double *GM, double *Y, double *mu, int *d_err,
                  cudaStream_t s) {
    if (k > NV_MAX) fail(GL_ERR_INVALID_ARG, "small_geneig: k too large");
    DBuf<double> work;
    work.alloc((size_t)n_sub * 3 * k * k);
    k_small_geneig<<<(n_sub + 63) / 64, 64, 0, s>>>(n_sub, k, GB, GM, Y, mu, d_err, work.p);
    GL_CUDA(cudaGetLastError());
    GL_CUDA(cudaStreamSynchronize(s));
}

// ---------------------------------------------------------------- rotations, scaling, random

__global__ void k_rotate(const int64_t *__restrict__ voff, const int64_t *__restrict__ vlen, const double *__restrict__ X,
                         const double *__restrict__ Y, int k, double *__restrict__ out) {
    const int s = blockIdx.x;
    const int64_t n = vlen[s], base = voff[s] * k;
    __shared__ double sy[NV_MAX * NV_MAX];
    for (int i = threadIdx.x; i < k * k; i += blockDim.x) sy[i] = Y[(int64_t)s * k * k + i];
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.y * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.y * blockDim.x) {
        double row[NV_MAX];
        for (int b = 0; b < k; ++b) row[b] = X[base + b * n + i];
        for (int a = 0; a < k; ++a) {
            double v = 0.0;
            for (int b = 0; b < k; ++b) v += row[b] * sy[b * k + a];
            out[base + a * n + i] = v;
        }
    }
}

void local_rotate(const FactorPlan &P, double *X, const double *Y, int k, double *tmp, cudaStream_t s) {
    dim3 g(P.n_sub, 64);
    k_rotate<<<g, 256, 0, s>>>(P.d_vec_off.p, P.d_vec_len.p, X, Y, k, tmp);
    GL_CUDA(cudaGetLastError());
    GL_CUDA(cudaMemcpyAsync(X, tmp, sizeof(double) * P.n_local * k, cudaMemcpyDeviceToDevice, s));
}

__global__ void k_scale_rows(const int64_t *__restrict__ voff, const int64_t *__restrict__ vlen, double *__restrict__ X,
                             const double *__restrict__ xi, int k) {
    const int s = blockIdx.x;
    const int64_t n = vlen[s], base = voff[s] * k;
    for (int64_t i = (int64_t)blockIdx.y * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.y * blockDim.x) {
        double w = xi[voff[s] + i];
        for (int a = 0; a < k; ++a) X[base + a * n + i] *= w;
    }
}

void scale_rows(const FactorPlan &P, double *X, const double *xi, int k, cudaStream_t s) {
    k_scale_rows<<<dim3(P.n_sub, 64), 256, 0, s>>>(P.d_vec_off.p, P.d_vec_len.p, X, xi, k);
    GL_CUDA(cudaGetLastError());
}

__global__ void k_fill_random(double *x, int64_t n, uint64_t seed) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint64_t z = seed + 0x9E3779B97F4A7C15ull * (uint64_t)(i + 1);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z = z ^ (z >> 31);
    x[i] = (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
}

void fill_random(double *x, int64_t n, uint64_t seed, cudaStream_t s) {
    if (!n) return;
    k_fill_random<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(x, n, seed);
    GL_CUDA(cudaGetLastError());
}

// ---------------------------------------------------------------- coarse restrict / prolong

__global__ void __launch_bounds__(256) k_coarse_restrict(const int64_t *__restrict__ voff, const int64_t *__restrict__ vlen,
                                                         const int64_t *__restrict__ gdof, const double *__restrict__ Z,
                                                         int m, const double *__restrict__ r, double *__restrict__ c) {
    const int s = blockIdx.x;
    const int64_t n = vlen[s], base = voff[s] * m;
    const int64_t *gd = gdof + voff[s];
    double acc[NV_MAX];
    for (int a = 0; a < m; ++a) acc[a] = 0.0;
    for (int64_t i = (int64_t)blockIdx.y * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.y * blockDim.x) {
        double ri = r[gd[i]];
        for (int a = 0; a < m; ++a) acc[a] += Z[base + a * n + i] * ri;
    }
    __shared__ double red[8][NV_MAX];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int a = 0; a < m; ++a) {
        double v = acc[a];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[w][a] = v;
    }
    __syncthreads();
    if (threadIdx.x < m) {
        double v = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) v += red[i][threadIdx.x];
        atomicAdd(c + (int64_t)s * m + threadIdx.x, v);
    }
}

void coarse_restrict(const FactorPlan &P, const double *Z, int m, const double *r, double *c, cudaStream_t s) {
    GL_CUDA(cudaMemsetAsync(c, 0, sizeof(double) * P.n_sub * m, s));
    k_coarse_restrict<<<dim3(P.n_sub, 32), 256, 0, s>>>(P.d_vec_off.p, P.d_vec_len.p, P.d_gdof.p, Z, m, r, c);
    GL_CUDA(cudaGetLastError());
}

__global__ void k_coarse_prolong(const int64_t *__restrict__ voff, const int64_t *__restrict__ vlen,
                                 const int64_t *__restrict__ gdof, const double *__restrict__ Z, int m,
                                 const double *__restrict__ y, double *__restrict__ z) {
    const int s = blockIdx.x;
    const int64_t n = vlen[s], base = voff[s] * m;
    const int64_t *gd = gdof + voff[s];
    __shared__ double sy[NV_MAX];
    if (threadIdx.x < m) sy[threadIdx.x] = y[(int64_t)s * m + threadIdx.x];
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.y * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.y * blockDim.x) {
        double v = 0.0;
        for (int a = 0; a < m; ++a) v += Z[base + a * n + i] * sy[a];
        atomicAdd(z + gd[i], v);
    }
}

void coarse_prolong(const FactorPlan &P, const double *Z, int m, const double *y, double *z, cudaStream_t s) {
    k_coarse_prolong<<<dim3(P.n_sub, 32), 256, 0, s>>>(P.d_vec_off.p, P.d_vec_len.p, P.d_gdof.p, Z, m, y, z);
    GL_CUDA(cudaGetLastError());
}

// ---------------------------------------------------------------- PCG vector kernels

constexpr int RED_BLOCKS = 1024;

__device__ __forceinline__ double block_sum(double v) {
    __shared__ double red[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    double t = 0.0;
    if (w == 0) {
        t = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    }
    return t;
}

__global__ void __launch_bounds__(256) k_dot_partial(const double *__restrict__ a, const double *__restrict__ b, int64_t n,
                                                     double *__restrict__ partials) {
    double v = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        v += a[i] * b[i];
    v = block_sum(v);
    if (threadIdx.x == 0) partials[blockIdx.x] = v;
}

__global__ void __launch_bounds__(1024) k_reduce_final(const double *__restrict__ partials, int n, double *__restrict__ out) {
    double v = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) v += partials[i];
    v = block_sum(v);
    if (threadIdx.x == 0) *out = v;
}

void dot(const double *a, const double *b, int64_t n, double *partials, double *out, cudaStream_t s) {
    k_dot_partial<<<RED_BLOCKS, 256, 0, s>>>(a, b, n, partials);
    k_reduce_final<<<1, 1024, 0, s>>>(partials, RED_BLOCKS, out);
    GL_CUDA(cudaGetLastError());
}

__global__ void __launch_bounds__(256) k_update_xr(double *__restrict__ x, double *__restrict__ r,
                                                   const double *__restrict__ p, const double *__restrict__ q, int64_t n,
                                                   CGScalars *__restrict__ S, double *__restrict__ partials) {
    const double alpha = S->rho / S->pq;
    double v = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        x[i] += alpha * p[i];
        double ri = r[i] - alpha * q[i];
        r[i] = ri;
        v += ri * ri;
    }
    v = block_sum(v);
    if (threadIdx.x == 0) partials[blockIdx.x] = v;
    if (blockIdx.x == 0 && threadIdx.x == 0) S->alpha = alpha;
}

void cg_update_xr(double *x, double *r, const double *p, const double *q, int64_t n, CGScalars *S, double *partials,
                  cudaStream_t s) {
    k_update_xr<<<RED_BLOCKS, 256, 0, s>>>(x, r, p, q, n, S, partials);
    k_reduce_final<<<1, 1024, 0, s>>>(partials, RED_BLOCKS, &S->rr);
    GL_CUDA(cudaGetLastError());
}

// beta = (rho_new - rz_old) / rho  (rz_old = 0 gives the standard recurrence)
__global__ void __launch_bounds__(256) k_update_p(double *__restrict__ p, const double *__restrict__ z, int64_t n,
                                                  CGScalars *__restrict__ S) {
    const double beta = (S->rho_new - S->rz_old) / S->rho;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = z[i] + beta * p[i];
}

__global__ void k_finish_p(CGScalars *S) {
    S->beta = (S->rho_new - S->rz_old) / S->rho;
    S->rho = S->rho_new;
}

// ---- per-part (segmented) versions for many laminates solved together

__global__ void __launch_bounds__(256) k_seg_dot(const double *__restrict__ a, const double *__restrict__ b,
                                                 const PartDesc *__restrict__ parts, double *__restrict__ partials) {
    const PartDesc pd = parts[blockIdx.x];
    double v = 0.0;
    for (int64_t i = (int64_t)blockIdx.y * blockDim.x + threadIdx.x; i < pd.n_dof; i += (int64_t)gridDim.y * blockDim.x)
        v += a[pd.dof_off + i] * b[pd.dof_off + i];
    v = block_sum(v);
    if (threadIdx.x == 0) partials[blockIdx.x * SEG_BLOCKS + blockIdx.y] = v;
}

__global__ void k_seg_final(const double *__restrict__ partials, double *__restrict__ out) {
    const int lane = threadIdx.x;   // 64 threads
    double v = partials[blockIdx.x * SEG_BLOCKS + lane];
    v += __shfl_xor_sync(0xffffffffu, v, 16);
    v += __shfl_xor_sync(0xffffffffu, v, 8);
    v += __shfl_xor_sync(0xffffffffu, v, 4);
    v += __shfl_xor_sync(0xffffffffu, v, 2);
    v += __shfl_xor_sync(0xffffffffu, v, 1);
    __shared__ double w[2];
    if ((lane & 31) == 0) w[lane >> 5] = v;
    __syncthreads();
    if (lane == 0) out[blockIdx.x] = w[0] + w[1];
}

void seg_dot(const double *a, const double *b, const PartDesc *parts, int n, double *partials, double *out,
             cudaStream_t s) {
    k_seg_dot<<<dim3(n, SEG_BLOCKS), 256, 0, s>>>(a, b, parts, partials);
    k_seg_final<<<n, SEG_BLOCKS, 0, s>>>(partials, out);
    GL_CUDA(cudaGetLastError());
}

__global__ void __launch_bounds__(256) k_seg_update_xr(double *__restrict__ x, double *__restrict__ r,
                                                       const double *__restrict__ p, const double *__restrict__ q,
                                                       const PartDesc *__restrict__ parts, SegScalars S,
                                                       double *__restrict__ partials) {
    const int ip = blockIdx.x;
    const PartDesc pd = parts[ip];
    const double alpha = S.active[ip] ? S.rho[ip] / S.pq[ip] : 0.0;
    double v = 0.0;
    for (int64_t i = (int64_t)blockIdx.y * blockDim.x + threadIdx.x; i < pd.n_dof; i += (int64_t)gridDim.y * blockDim.x) {
        const int64_t g = pd.dof_off + i;
        x[g] += alpha * p[g];
        const double ri = r[g] - alpha * q[g];
        r[g] = ri;
        v += ri * ri;
    }
    v = block_sum(v);
    if (threadIdx.x == 0) partials[ip * SEG_BLOCKS + blockIdx.y] = v;
}

void seg_update_xr(double *x, double *r, const double *p, const double *q, const PartDesc *parts, int n,
                   SegScalars S, double *partials, cudaStream_t s) {
    k_seg_update_xr<<<dim3(n, SEG_BLOCKS), 256, 0, s>>>(x, r, p, q, parts, S, partials);
    k_seg_final<<<n, SEG_BLOCKS, 0, s>>>(partials, S.rr);
    GL_CUDA(cudaGetLastError());
}

__global__ void __launch_bounds__(256) k_seg_update_p(double *__restrict__ p, const double *__restrict__ z,
                                                      const PartDesc *__restrict__ parts, SegScalars S) {
    const int ip = blockIdx.x;
    const PartDesc pd = parts[ip];
    const double rho = S.rho[ip];
    const double beta = rho != 0.0 ? (S.rho_new[ip] - S.rz_old[ip]) / rho : 0.0;
    for (int64_t i = (int64_t)blockIdx.y * blockDim.x + threadIdx.x; i < pd.n_dof; i += (int64_t)gridDim.y * blockDim.x) {
        const int64_t g = pd.dof_off + i;
        p[g] = z[g] + beta * p[g];
    }
}

__global__ void k_seg_rho(SegScalars S, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) S.rho[i] = S.rho_new[i];
}

void seg_update_p(double *p, const double *z, const PartDesc *parts, int n, SegScalars S, cudaStream_t s) {
    k_seg_update_p<<<dim3(n, SEG_BLOCKS), 256, 0, s>>>(p, z, parts, S);
    k_seg_rho<<<(n + 127) / 128, 128, 0, s>>>(S, n);
    GL_CUDA(cudaGetLastError());
}

__global__ void k_seg_check(SegScalars S, int n, double tol2, int max_iter, int *n_active) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || !S.active[i]) return;
    const int it = ++S.iters[i];
    const double rr = S.rr[i];
    int a = 1;
    if (!(rr > tol2 * S.ff[i]) || it >= max_iter) a = 0;   // converged, stalled at max_iter, or NaN
    S.active[i] = a;
    if (a) atomicAdd(n_active, 1);
}

void seg_check(SegScalars S, int n, double tol, int max_iter, int *n_active, cudaStream_t s) {
    GL_CUDA(cudaMemsetAsync(n_active, 0, sizeof(int), s));
    k_seg_check<<<(n + 127) / 128, 128, 0, s>>>(S, n, tol * tol, max_iter, n_active);
    GL_CUDA(cudaGetLastError());
}

__global__ void k_seg_confirm(SegScalars S, int n, double tol2, int max_iter, int *n_active) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || S.active[i] || !(S.ff[i] > 0.0) || S.iters[i] >= max_iter) return;
    const double rr = S.rr[i];
    if (rr > tol2 * S.ff[i] && rr < INFINITY) {
        S.active[i] = 1;
        atomicAdd(n_active, 1);
    }
}

void seg_confirm(SegScalars S, int n, double tol, int max_iter, int *n_active, cudaStream_t s) {
    GL_CUDA(cudaMemsetAsync(n_active, 0, sizeof(int), s));
    k_seg_confirm<<<(n + 127) / 128, 128, 0, s>>>(S, n, tol * tol, max_iter, n_active);
    GL_CUDA(cudaGetLastError());
}

void cg_update_p(double *p, const double *z, int64_t n, CGScalars *S, cudaStream_t s) {
    k_update_p<<<RED_BLOCKS, 256, 0, s>>>(p, z, n, S);
    k_finish_p<<<1, 1, 0, s>>>(S);
    GL_CUDA(cudaGetLastError());
}

__global__ void k_set_entries(double *__restrict__ y, const int64_t *__restrict__ dof, int64_t n,
                              const double *__restrict__ vals) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) y[dof[i]] = vals ? vals[i] : 0.0;
}

void set_entries(double *y, const int64_t *dof, int64_t n, const double *vals, cudaStream_t s) {
    if (!n) return;
    k_set_entries<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(y, dof, n, vals);
    GL_CUDA(cudaGetLastError());
}

__global__ void k_sub(double *__restrict__ y, const double *__restrict__ a, const double *__restrict__ b, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = a[i] - b[i];
}

void sub(double *y, const double *a, const double *b, int64_t n, cudaStream_t s) {
    k_sub<<<RED_BLOCKS, 256, 0, s>>>(y, a, b, n);
    GL_CUDA(cudaGetLastError());
}

__global__ void k_axpy(double *__restrict__ y, double a, const double *__restrict__ x, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] += a * x[i];
}

void axpy(double *y, double a, const double *x, int64_t n, cudaStream_t s) {
    k_axpy<<<RED_BLOCKS, 256, 0, s>>>(y, a, x, n);
    GL_CUDA(cudaGetLastError());
}

__global__ void k_max_where(const double *__restrict__ v, const uint8_t *__restrict__ mask, int64_t n,
                            double *__restrict__ out) {
    __shared__ double red[256];
    double m = -1e300;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x)
        if (mask[i]) m = fmax(m, v[i]);
    red[threadIdx.x] = m;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0];
}

void max_where(const double *v, const uint8_t *mask, int64_t n, double *out, cudaStream_t s) {
    k_max_where<<<1, 256, 0, s>>>(v, mask, n, out);
    GL_CUDA(cudaGetLastError());
}

}  // namespace gl
