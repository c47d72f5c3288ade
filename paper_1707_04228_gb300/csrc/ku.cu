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
// block.  The whole product is FP64-ALU bound on this part (about 2k FMA per
// element per direction of the contractions plus ~100 FMA per Gauss point).
#include "gl_internal.h"
#include "q2.cuh"

namespace gl {

constexpr int KU_EPB = 4;

__global__ void __launch_bounds__(32 * KU_EPB) k_ku(int64_t n_elem, int nx, int ny, int NX, int NY,
                                                   const double *__restrict__ C, const double *__restrict__ geo,
                                                   const double *__restrict__ x, double *__restrict__ y) {
    __shared__ double sU[KU_EPB][3][27];
    __shared__ double sA[KU_EPB][3][27];
    __shared__ double sB[KU_EPB][3][27];
    __shared__ double sAA[KU_EPB][3][27];
    __shared__ double sAB[KU_EPB][3][27];
    __shared__ double sBA[KU_EPB][3][27];
    __shared__ double sC[KU_EPB][36];
    const int w = threadIdx.x >> 5, t = threadIdx.x & 31;
    const int64_t e = (int64_t)blockIdx.x * KU_EPB + w;
    if (e >= n_elem) return;   // whole warp leaves together
    Q2Tables T;
    T.init();
    const int ex = (int)(e % nx), ey = (int)((e / nx) % ny), ez = (int)(e / ((int64_t)nx * ny));
    const bool on = t < 27;
    const int ti = t % 3, tj = (t / 3) % 3, tk = t / 9;   // lane as (i, j, k) or (qx, qy, qz)
    int64_t node = 0;
    if (on) {
        node = (int64_t)(2 * ex + ti) + (int64_t)NX * ((2 * ey + tj) + (int64_t)NY * (2 * ez + tk));
        sU[w][0][t] = x[3 * node + 0];
        sU[w][1][t] = x[3 * node + 1];
        sU[w][2][t] = x[3 * node + 2];
    }
    for (int i = t; i < 36; i += 32) sC[w][i] = C[36 * e + i];
    __syncwarp();
    // stage 1: contract i -> qx (lane = (qx, j, k))
    if (on) {
        for (int c = 0; c < 3; ++c) {
            const double *u = &sU[w][c][3 * tj + 9 * tk];
            sA[w][c][t] = T.N[ti][0] * u[0] + T.N[ti][1] * u[1] + T.N[ti][2] * u[2];
            sB[w][c][t] = T.D[ti][0] * u[0] + T.D[ti][1] * u[1] + T.D[ti][2] * u[2];
        }
    }
    __syncwarp();
    // stage 2: contract j -> qy (lane = (qx, qy, k))
    if (on) {
        for (int c = 0; c < 3; ++c) {
            const double *a = &sA[w][c][ti + 9 * tk];
            const double *b = &sB[w][c][ti + 9 * tk];
            sAA[w][c][t] = T.N[tj][0] * a[0] + T.N[tj][1] * a[3] + T.N[tj][2] * a[6];
            sAB[w][c][t] = T.D[tj][0] * a[0] + T.D[tj][1] * a[3] + T.D[tj][2] * a[6];
            sBA[w][c][t] = T.N[tj][0] * b[0] + T.N[tj][1] * b[3] + T.N[tj][2] * b[6];
        }
    }
    __syncwarp();
    // stage 3: contract k -> qz (lane = Gauss point (qx, qy, qz)), then the pointwise stress
    double F[3][3];
    if (on) {
        double G[3][3];
        for (int c = 0; c < 3; ++c) {
            const double *aa = &sAA[w][c][ti + 3 * tj];
            const double *ab = &sAB[w][c][ti + 3 * tj];
            const double *ba = &sBA[w][c][ti + 3 * tj];
            G[c][0] = T.N[tk][0] * ba[0] + T.N[tk][1] * ba[9] + T.N[tk][2] * ba[18];
            G[c][1] = T.N[tk][0] * ab[0] + T.N[tk][1] * ab[9] + T.N[tk][2] * ab[18];
            G[c][2] = T.D[tk][0] * aa[0] + T.D[tk][1] * aa[9] + T.D[tk][2] * aa[18];
        }
        const double *g = geo + 10 * (e * 27 + t);
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
        double s[6];
        const double *Ce = sC[w];
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            double v = 0.0;
#pragma unroll
            for (int j = 0; j < 6; ++j) v += Ce[6 * i + j] * eps[j];
            s[i] = v * wd;
        }
        const double S[3][3] = {{s[0], s[5], s[4]}, {s[5], s[1], s[3]}, {s[4], s[3], s[2]}};
        // reference flux F[c][e] = w |J| sum_d sigma_cd dxi_e/dx_d
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int r = 0; r < 3; ++r) F[c][r] = S[c][0] * Ji[3 * r + 0] + S[c][1] * Ji[3 * r + 1] + S[c][2] * Ji[3 * r + 2];
    }
    __syncwarp();
    if (on) {
        for (int c = 0; c < 3; ++c) {
            sAA[w][c][t] = F[c][0];
            sAB[w][c][t] = F[c][1];
            sBA[w][c][t] = F[c][2];
        }
    }
    __syncwarp();
    // stage 3^T: qz -> k (lane = (qx, qy, k))
    if (on) {
        for (int c = 0; c < 3; ++c) {
            const double *fx = &sAA[w][c][ti + 3 * tj];
            const double *fy = &sAB[w][c][ti + 3 * tj];
            const double *fz = &sBA[w][c][ti + 3 * tj];
            sA[w][c][t] = T.N[0][tk] * fx[0] + T.N[1][tk] * fx[9] + T.N[2][tk] * fx[18];
            sB[w][c][t] = T.N[0][tk] * fy[0] + T.N[1][tk] * fy[9] + T.N[2][tk] * fy[18];
            sU[w][c][t] = T.D[0][tk] * fz[0] + T.D[1][tk] * fz[9] + T.D[2][tk] * fz[18];
        }
    }
    __syncwarp();
    // stage 2^T: qy -> j (lane = (qx, j, k))
    if (on) {
        for (int c = 0; c < 3; ++c) {
            const double *px = &sA[w][c][ti + 9 * tk];
            const double *py = &sB[w][c][ti + 9 * tk];
            const double *pz = &sU[w][c][ti + 9 * tk];
            sAA[w][c][t] = T.N[0][tj] * px[0] + T.N[1][tj] * px[3] + T.N[2][tj] * px[6];
            sAB[w][c][t] = T.D[0][tj] * py[0] + T.D[1][tj] * py[3] + T.D[2][tj] * py[6] +
                           T.N[0][tj] * pz[0] + T.N[1][tj] * pz[3] + T.N[2][tj] * pz[6];
        }
    }
    __syncwarp();
    // stage 1^T: qx -> i (lane = node (i, j, k)) and scatter-add
    if (on) {
        for (int c = 0; c < 3; ++c) {
            const double *r1 = &sAA[w][c][3 * tj + 9 * tk];
            const double *r2 = &sAB[w][c][3 * tj + 9 * tk];
            double v = T.D[0][ti] * r1[0] + T.D[1][ti] * r1[1] + T.D[2][ti] * r1[2] + T.N[0][ti] * r2[0] +
                       T.N[1][ti] * r2[1] + T.N[2][ti] * r2[2];
            atomicAdd(y + 3 * node + c, v);
        }
    }
}

void launch_ku(const MeshHost &m, const double *C, const double *geo, const double *x, double *y, cudaStream_t s) {
    GL_CUDA(cudaMemsetAsync(y, 0, m.n_dof * sizeof(double), s));
    int64_t nb = (m.n_elem + KU_EPB - 1) / KU_EPB;
    k_ku<<<(unsigned)nb, 32 * KU_EPB, 0, s>>>(m.n_elem, m.nx, m.ny, m.NX, m.NY, C, geo, x, y);
    GL_CUDA(cudaGetLastError());
}

}  // namespace gl
