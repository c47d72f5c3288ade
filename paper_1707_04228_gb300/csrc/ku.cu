// Matrix-free element-by-element K u for Q2 hexahedra in FP64 (Section 2.3:
// the iterative solver only needs products with the sparse stiffness K).
//
// y = sum_e P_e^T K_e P_e x with K_e = sum_q w_q |J_q| B_q^T C_e B_q (full
// 3x3x3 Gauss integration), never forming K_e: per element the 27x3 nodal
// values are gathered into shared memory, reference gradients at the 27 Gauss
// points come from three sum-factorised 1D contractions, the stress
// sigma = C_e eps is formed pointwise, and the transposed contractions give
// the 81 element residual entries, scatter-added with FP64 atomics.
//
// One 32-lane warp per element (27 active lanes: lane t is node t in the
// gather/scatter, Gauss point t in the pointwise stage); EPB elements per
// block.  The product is FP64-ALU bound on this part (6,318 FMA per element
// against 2,448 B of element data and 16 B per DOF of vector traffic).
//
// The same element core serves the global product (node-major global
// vectors) and the subdomain-local products of the GenEO setup (local
// vectors reached through per-element index maps, optional diagonal
// scaling on both sides, several vectors per call).
#include "geneo.h"
#include "q2.cuh"

namespace gl {

constexpr int KU_EPB = 4;

struct KuSmem {
    double U[3][27], A[3][27], B[3][27], AA[3][27], AB[3][27], BA[3][27], C[36];
};

// Element residual of the values in s.U (component-major, node t = i + 3j + 9k).
// On return lane t (< 27) holds the three components of node t in out[].
__device__ __forceinline__ void ku_core(KuSmem &s, const Q2Tables &T, int t, const double *__restrict__ geo_e,
                                        double out[3]) {
    const bool on = t < 27;
    const int ti = t % 3, tj = (t / 3) % 3, tk = t / 9;
    // stage 1: contract i -> qx (lane = (qx, j, k))
    if (on) {
        for (int c = 0; c < 3; ++c) {
            const double *u = &s.U[c][3 * tj + 9 * tk];
            s.A[c][t] = T.N[ti][0] * u[0] + T.N[ti][1] * u[1] + T.N[ti][2] * u[2];
            s.B[c][t] = T.D[ti][0] * u[0] + T.D[ti][1] * u[1] + T.D[ti][2] * u[2];
        }
    }
    __syncwarp();
    // stage 2: contract j -> qy (lane = (qx, qy, k))
    if (on) {
        for (int c = 0; c < 3; ++c) {
            const double *a = &s.A[c][ti + 9 * tk];
            const double *b = &s.B[c][ti + 9 * tk];
            s.AA[c][t] = T.N[tj][0] * a[0] + T.N[tj][1] * a[3] + T.N[tj][2] * a[6];
            s.AB[c][t] = T.D[tj][0] * a[0] + T.D[tj][1] * a[3] + T.D[tj][2] * a[6];
            s.BA[c][t] = T.N[tj][0] * b[0] + T.N[tj][1] * b[3] + T.N[tj][2] * b[6];
        }
    }
    __syncwarp();
    // stage 3: contract k -> qz (lane = Gauss point), pointwise stress and reference flux
    double F[3][3];
    if (on) {
        double G[3][3];
        for (int c = 0; c < 3; ++c) {
            const double *aa = &s.AA[c][ti + 3 * tj];
            const double *ab = &s.AB[c][ti + 3 * tj];
            const double *ba = &s.BA[c][ti + 3 * tj];
            G[c][0] = T.N[tk][0] * ba[0] + T.N[tk][1] * ba[9] + T.N[tk][2] * ba[18];
            G[c][1] = T.N[tk][0] * ab[0] + T.N[tk][1] * ab[9] + T.N[tk][2] * ab[18];
            G[c][2] = T.D[tk][0] * aa[0] + T.D[tk][1] * aa[9] + T.D[tk][2] * aa[18];
        }
        const double *g = geo_e + 10 * t;
        double Ji[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) Ji[i] = g[i];
        const double wd = g[9];
        double H[3][3];
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int d = 0; d < 3; ++d) H[c][d] = G[c][0] * Ji[0 + d] + G[c][1] * Ji[3 + d] + G[c][2] * Ji[6 + d];
        const double eps[6] = {H[0][0], H[1][1], H[2][2], H[1][2] + H[2][1], H[0][2] + H[2][0], H[0][1] + H[1][0]};
        double sv[6];
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            double v = 0.0;
#pragma unroll
            for (int j = 0; j < 6; ++j) v += s.C[6 * i + j] * eps[j];
            sv[i] = v * wd;
        }
        const double S[3][3] = {{sv[0], sv[5], sv[4]}, {sv[5], sv[1], sv[3]}, {sv[4], sv[3], sv[2]}};
        // reference flux F[c][r] = w |J| sum_d sigma_cd dxi_r/dx_d
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int r = 0; r < 3; ++r) F[c][r] = S[c][0] * Ji[3 * r + 0] + S[c][1] * Ji[3 * r + 1] + S[c][2] * Ji[3 * r + 2];
    }
    __syncwarp();
    if (on) {
        for (int c = 0; c < 3; ++c) {
            s.AA[c][t] = F[c][0];
            s.AB[c][t] = F[c][1];
            s.BA[c][t] = F[c][2];
        }
    }
    __syncwarp();
    // stage 3^T: qz -> k (lane = (qx, qy, k))
    if (on) {
        for (int c = 0; c < 3; ++c) {
            const double *fx = &s.AA[c][ti + 3 * tj];
            const double *fy = &s.AB[c][ti + 3 * tj];
            const double *fz = &s.BA[c][ti + 3 * tj];
            s.A[c][t] = T.N[0][tk] * fx[0] + T.N[1][tk] * fx[9] + T.N[2][tk] * fx[18];
            s.B[c][t] = T.N[0][tk] * fy[0] + T.N[1][tk] * fy[9] + T.N[2][tk] * fy[18];
            s.U[c][t] = T.D[0][tk] * fz[0] + T.D[1][tk] * fz[9] + T.D[2][tk] * fz[18];
        }
    }
    __syncwarp();
    // stage 2^T: qy -> j (lane = (qx, j, k))
    if (on) {
        for (int c = 0; c < 3; ++c) {
            const double *px = &s.A[c][ti + 9 * tk];
            const double *py = &s.B[c][ti + 9 * tk];
            const double *pz = &s.U[c][ti + 9 * tk];
            s.AA[c][t] = T.N[0][tj] * px[0] + T.N[1][tj] * px[3] + T.N[2][tj] * px[6];
            s.AB[c][t] = T.D[0][tj] * py[0] + T.D[1][tj] * py[3] + T.D[2][tj] * py[6] + T.N[0][tj] * pz[0] +
                         T.N[1][tj] * pz[3] + T.N[2][tj] * pz[6];
        }
    }
    __syncwarp();
    // stage 1^T: qx -> i (lane = node (i, j, k))
    if (on) {
        for (int c = 0; c < 3; ++c) {
            const double *r1 = &s.AA[c][3 * tj + 9 * tk];
            const double *r2 = &s.AB[c][3 * tj + 9 * tk];
            out[c] = T.D[0][ti] * r1[0] + T.D[1][ti] * r1[1] + T.D[2][ti] * r1[2] + T.N[0][ti] * r2[0] +
                     T.N[1][ti] * r2[1] + T.N[2][ti] * r2[2];
        }
    }
    __syncwarp();
}

__global__ void __launch_bounds__(32 * KU_EPB) k_ku(int64_t n_elem, int nx, int ny, int NX, int NY,
                                                   const double *__restrict__ C, const double *__restrict__ geo,
                                                   const double *__restrict__ x, double *__restrict__ y) {
    __shared__ KuSmem sm[KU_EPB];
    const int w = threadIdx.x >> 5, t = threadIdx.x & 31;
    const int64_t e = (int64_t)blockIdx.x * KU_EPB + w;
    if (e >= n_elem) return;   // whole warp leaves together
    KuSmem &s = sm[w];
    Q2Tables T;
    T.init();
    const int ex = (int)(e % nx), ey = (int)((e / nx) % ny), ez = (int)(e / ((int64_t)nx * ny));
    int64_t node = 0;
    if (t < 27) {
        node = (int64_t)(2 * ex + t % 3) + (int64_t)NX * ((2 * ey + (t / 3) % 3) + (int64_t)NY * (2 * ez + t / 9));
        s.U[0][t] = x[3 * node + 0];
        s.U[1][t] = x[3 * node + 1];
        s.U[2][t] = x[3 * node + 2];
    }
    for (int i = t; i < 36; i += 32) s.C[i] = C[36 * e + i];
    __syncwarp();
    double out[3];
    ku_core(s, T, t, geo + 270 * e, out);
    if (t < 27) {
        atomicAdd(y + 3 * node + 0, out[0]);
        atomicAdd(y + 3 * node + 1, out[1]);
        atomicAdd(y + 3 * node + 2, out[2]);
    }
}

void launch_ku(const MeshHost &m, const double *C, const double *geo, const double *x, double *y, cudaStream_t s) {
    GL_CUDA(cudaMemsetAsync(y, 0, m.n_dof * sizeof(double), s));
    int64_t nb = (m.n_elem + KU_EPB - 1) / KU_EPB;
    k_ku<<<(unsigned)nb, 32 * KU_EPB, 0, s>>>(m.n_elem, m.nx, m.ny, m.NX, m.NY, C, geo, x, y);
    GL_CUDA(cudaGetLastError());
}

// Many laminates in one launch: elements of all parts are numbered
// consecutively (part i owns [elem_off[i], elem_off[i+1])), C and geo are
// indexed by that global id, and part i's DOFs start at dof_off[i] of the
// concatenated vectors.  Each warp finds its part by binary search.
__global__ void __launch_bounds__(32 * KU_EPB) k_ku_batch(const PartDesc *__restrict__ parts, int n_parts,
                                                         int64_t n_elem, const double *__restrict__ C,
                                                         const double *__restrict__ geo, const double *__restrict__ x,
                                                         double *__restrict__ y) {
    __shared__ KuSmem sm[KU_EPB];
    const int w = threadIdx.x >> 5, t = threadIdx.x & 31;
    const int64_t eg = (int64_t)blockIdx.x * KU_EPB + w;
    if (eg >= n_elem) return;
    int lo = 0, hi = n_parts - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (parts[mid].elem_off <= eg) lo = mid;
        else hi = mid - 1;
    }
    const PartDesc pd = parts[lo];
    const int64_t e = eg - pd.elem_off;
    KuSmem &s = sm[w];
    Q2Tables T;
    T.init();
    const int ex = (int)(e % pd.nx), ey = (int)((e / pd.nx) % pd.ny), ez = (int)(e / ((int64_t)pd.nx * pd.ny));
    int64_t dof = 0;
    if (t < 27) {
        int64_t node = (int64_t)(2 * ex + t % 3) +
                       (int64_t)pd.NX * ((2 * ey + (t / 3) % 3) + (int64_t)pd.NY * (2 * ez + t / 9));
        dof = pd.dof_off + 3 * node;
        s.U[0][t] = x[dof + 0];
        s.U[1][t] = x[dof + 1];
        s.U[2][t] = x[dof + 2];
    }
    for (int i = t; i < 36; i += 32) s.C[i] = C[36 * eg + i];
    __syncwarp();
    double out[3];
    ku_core(s, T, t, geo + 270 * eg, out);
    if (t < 27) {
        atomicAdd(y + dof + 0, out[0]);
        atomicAdd(y + dof + 1, out[1]);
        atomicAdd(y + dof + 2, out[2]);
    }
}

void launch_ku_batch(const PartDesc *d_parts, int n_parts, int64_t n_elem, int64_t n_dof, const double *C,
                     const double *geo, const double *x, double *y, cudaStream_t s) {
    GL_CUDA(cudaMemsetAsync(y, 0, n_dof * sizeof(double), s));
    int64_t nb = (n_elem + KU_EPB - 1) / KU_EPB;
    k_ku_batch<<<(unsigned)nb, 32 * KU_EPB, 0, s>>>(d_parts, n_parts, n_elem, C, geo, x, y);
    GL_CUDA(cudaGetLastError());
}

// Subdomain-local products y_s += S K_s S x_s for nv vectors per subdomain
// (S = diag(xi) or identity), through the element -> local index maps.
__global__ void __launch_bounds__(32 * KU_EPB) k_local_ku(int64_t n_pairs, const int *__restrict__ elem,
                                                         const int *__restrict__ sub, const int *__restrict__ loc,
                                                         const int64_t *__restrict__ voff,
                                                         const int64_t *__restrict__ vlen,
                                                         const double *__restrict__ C, const double *__restrict__ geo,
                                                         const double *__restrict__ xi, const double *__restrict__ x,
                                                         double *__restrict__ y, int nv) {
    __shared__ KuSmem sm[KU_EPB];
    const int w = threadIdx.x >> 5, t = threadIdx.x & 31;
    const int64_t pi = (int64_t)blockIdx.x * KU_EPB + w;
    if (pi >= n_pairs) return;
    KuSmem &s = sm[w];
    Q2Tables T;
    T.init();
    const int64_t e = elem[pi];
    const int sb = sub[pi];
    const int64_t base = voff[sb] * nv, n = vlen[sb];
    int l[3] = {-1, -1, -1};
    double sc[3] = {0, 0, 0};
    if (t < 27)
        for (int c = 0; c < 3; ++c) {
            l[c] = loc[pi * 81 + 3 * t + c];
            sc[c] = l[c] >= 0 ? (xi ? xi[voff[sb] + l[c]] : 1.0) : 0.0;
        }
    for (int i = t; i < 36; i += 32) s.C[i] = C[36 * e + i];
    for (int v = 0; v < nv; ++v) {
        if (t < 27)
            for (int c = 0; c < 3; ++c) s.U[c][t] = l[c] >= 0 ? x[base + (int64_t)v * n + l[c]] * sc[c] : 0.0;
        __syncwarp();
        double out[3];
        ku_core(s, T, t, geo + 270 * e, out);
        if (t < 27)
            for (int c = 0; c < 3; ++c)
                if (l[c] >= 0) atomicAdd(y + base + (int64_t)v * n + l[c], out[c] * sc[c]);
        __syncwarp();
    }
}

void local_K_apply(const FactorPlan &P, const LocalElems &E, const double *C, const double *geo, const double *xi,
                   const double *x, double *y, int nv, cudaStream_t s) {
    if (!E.n_pairs) return;
    int64_t nb = (E.n_pairs + KU_EPB - 1) / KU_EPB;
    k_local_ku<<<(unsigned)nb, 32 * KU_EPB, 0, s>>>(E.n_pairs, E.elem.p, E.sub.p, E.loc.p, P.d_vec_off.p,
                                                   P.d_vec_len.p, C, geo, xi, x, y, nv);
    GL_CUDA(cudaGetLastError());
}

}  // namespace gl
