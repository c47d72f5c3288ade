// Adjoint pieces for gradients with respect to the per-element fibre
// misalignment angles theta_e.
//
// For an objective J(sigma(u, theta), theta) with K(theta) u = f on the free
// DOFs: dJ/dtheta_e = dJ/dtheta_e|_u - lambda_e^T (dK_e/dtheta_e) u_e, where
// K_ff lambda = (dJ/du)_f and lambda = 0 on Dirichlet DOFs.  dK_e/dtheta_e =
// sum_q w_q |J_q| B_q^T (dC_e/dtheta_e) B_q, and C_e = M C_mat M^T with M the
// Bond matrix of R = R_l(psi + theta) R_r(phi), so dC = dM C M^T + M C dM^T.
#include "gl_internal.h"
#include "q2.cuh"

namespace gl {

namespace {

__device__ void bond_pair(const double a[3][3], const double da[3][3], double M[6][6], double dM[6][6]) {
    const int I0[6] = {0, 1, 2, 1, 0, 0}, I1[6] = {0, 1, 2, 2, 2, 1};
    for (int r = 0; r < 6; ++r) {
        int i = I0[r], j = I1[r];
        for (int c = 0; c < 6; ++c) {
            int k = I0[c], l = I1[c];
            double v = a[i][k] * a[j][l], dv = da[i][k] * a[j][l] + a[i][k] * da[j][l];
            if (k != l) {
                v += a[i][l] * a[j][k];
                dv += da[i][l] * a[j][k] + a[i][l] * da[j][k];
            }
            M[r][c] = v;
            dM[r][c] = dv;
        }
    }
}

// dC_e/dtheta_e (6x6, global axes) for element e.
__device__ void dC_dtheta(int64_t e, int nx, int ny, const int *layer_of_ez, const int *layer_mat,
                          const int *elem_mat, const double *layer_angle, const double *theta, const double *psi_x,
                          const double *matC, double dC[6][6]) {
    int ex = (int)(e % nx);
    int ez = (int)(e / ((int64_t)nx * ny));
    int layer = layer_of_ez[ez];
    const double *Cm = matC + 36 * (elem_mat ? elem_mat[e] : layer_mat[layer]);
    double phi = layer_angle[layer];
    double a = psi_x[ex] + (theta ? theta[e] : 0.0);
    double ca = cos(a), sa = sin(a), cp = cos(phi), sp = sin(phi);
    double Ry[3][3] = {{ca, 0, sa}, {0, 1, 0}, {-sa, 0, ca}};
    double dRy[3][3] = {{-sa, 0, ca}, {0, 0, 0}, {-ca, 0, -sa}};
    double Rz[3][3] = {{cp, -sp, 0}, {sp, cp, 0}, {0, 0, 1}};
    double R[3][3], dR[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double v = 0, dv = 0;
            for (int k = 0; k < 3; ++k) {
                v += Ry[i][k] * Rz[k][j];
                dv += dRy[i][k] * Rz[k][j];
            }
            R[i][j] = v;
            dR[i][j] = dv;
        }
    double M[6][6], dM[6][6];
    bond_pair(R, dR, M, dM);
    double T1[6][6], T2[6][6];   // T1 = dM C, T2 = M C
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) {
            double v1 = 0, v2 = 0;
            for (int k = 0; k < 6; ++k) {
                v1 += dM[i][k] * Cm[6 * k + j];
                v2 += M[i][k] * Cm[6 * k + j];
            }
            T1[i][j] = v1;
            T2[i][j] = v2;
        }
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) {
            double v = 0;
            for (int k = 0; k < 6; ++k) v += T1[i][k] * M[j][k] + T2[i][k] * dM[j][k];
            dC[i][j] = v;
        }
}

__device__ __forceinline__ int64_t node_of(int ex, int ey, int ez, int a, int NX, int NY) {
    return (int64_t)(2 * ex + a % 3) + (int64_t)NX * ((2 * ey + (a / 3) % 3) + (int64_t)NY * (2 * ez + a / 9));
}

__device__ void inv3(const double J[3][3], double Ji[3][3]) {
    double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) - J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                 J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
    double id = 1.0 / det;
    Ji[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) * id;
    Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) * id;
    Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) * id;
    Ji[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) * id;
    Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) * id;
    Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) * id;
    Ji[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) * id;
    Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) * id;
    Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) * id;
}

}  // namespace

// Vector-Jacobian product of the centre stress recovery (s33 = sigma_rr,
// t13 = tau_rs in the (s,l,r) frame): dJdu += sum_e (w33_e ds33_e/du +
// w13_e dt13_e/du); dJdth[e] = w33_e ds33_e/dtheta_e + w13_e dt13_e/dtheta_e at
// fixed u.  One thread per element.
__global__ void k_stress_vjp(int64_t n_elem, int nx, int ny, int NX, int NY, const double *__restrict__ X,
                             const double *__restrict__ C, const double *__restrict__ psi_x,
                             const int *__restrict__ layer_of_ez, const int *__restrict__ layer_mat,
                             const int *__restrict__ elem_mat, const double *__restrict__ layer_angle,
                             const double *__restrict__ theta, const double *__restrict__ matC,
                             const double *__restrict__ u,
                             const double *__restrict__ w33, const double *__restrict__ w13,
                             double *__restrict__ dJdu, double *__restrict__ dJdth) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n_elem) return;
    const double a33 = w33 ? w33[e] : 0.0, a13 = w13 ? w13[e] : 0.0;
    if (a33 == 0.0 && a13 == 0.0) {
        if (dJdth) dJdth[e] = 0.0;
        return;
    }
    int ex = (int)(e % nx), ey = (int)((e / nx) % ny), ez = (int)(e / ((int64_t)nx * ny));
    const int I0[6] = {0, 1, 2, 1, 0, 0}, I1[6] = {0, 1, 2, 2, 2, 1};
    double Rf[3][3];
    rot_width(psi_x[ex], Rf);
    // s33 = sum_ij Rf[i][2] Rf[j][2] S_ij, t13 = sum_ij Rf[i][0] Rf[j][2] S_ij; in Voigt weights
    double wv[6];
    for (int I = 0; I < 6; ++I) {
        int i = I0[I], j = I1[I];
        double v33 = Rf[i][2] * Rf[j][2], v13 = Rf[i][0] * Rf[j][2];
        if (i != j) {
            v33 += Rf[j][2] * Rf[i][2];
            v13 += Rf[j][0] * Rf[i][2];
        }
        wv[I] = a33 * v33 + a13 * v13;
    }
    // centre Jacobian and strain
    double J[3][3] = {{0}}, G[3][3] = {{0}}, dN[27][3];
    for (int a = 0; a < 27; ++a) {
        int i = a % 3, j = (a / 3) % 3, k = a / 9;
        dN[a][0] = q2_dN(i, 0.0) * q2_N(j, 0.0) * q2_N(k, 0.0);
        dN[a][1] = q2_N(i, 0.0) * q2_dN(j, 0.0) * q2_N(k, 0.0);
        dN[a][2] = q2_N(i, 0.0) * q2_N(j, 0.0) * q2_dN(k, 0.0);
        if (dN[a][0] == 0.0 && dN[a][1] == 0.0 && dN[a][2] == 0.0) continue;
        int64_t n = node_of(ex, ey, ez, a, NX, NY);
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) {
                J[r][c] += X[3 * n + r] * dN[a][c];
                G[r][c] += u[3 * n + r] * dN[a][c];
            }
    }
    double Ji[3][3];
    inv3(J, Ji);
    const double *Ce = C + 36 * e;
    double g[6];   // C^T wv (C symmetric)
    for (int I = 0; I < 6; ++I) {
        double v = 0;
        for (int K = 0; K < 6; ++K) v += Ce[6 * K + I] * wv[K];
        g[I] = v;
    }
    if (dJdu) {
        for (int a = 0; a < 27; ++a) {
            if (dN[a][0] == 0.0 && dN[a][1] == 0.0 && dN[a][2] == 0.0) continue;
            double dx = 0, dy = 0, dz = 0;
            for (int q = 0; q < 3; ++q) {
                dx += dN[a][q] * Ji[q][0];
                dy += dN[a][q] * Ji[q][1];
                dz += dN[a][q] * Ji[q][2];
            }
            int64_t n = node_of(ex, ey, ez, a, NX, NY);
            atomicAdd(dJdu + 3 * n + 0, g[0] * dx + g[4] * dz + g[5] * dy);
            atomicAdd(dJdu + 3 * n + 1, g[1] * dy + g[3] * dz + g[5] * dx);
            atomicAdd(dJdu + 3 * n + 2, g[2] * dz + g[3] * dy + g[4] * dx);
        }
    }
    if (dJdth) {
        double H[3][3];
        for (int c = 0; c < 3; ++c)
            for (int d = 0; d < 3; ++d) H[c][d] = G[c][0] * Ji[0][d] + G[c][1] * Ji[1][d] + G[c][2] * Ji[2][d];
        double eps[6] = {H[0][0], H[1][1], H[2][2], H[1][2] + H[2][1], H[0][2] + H[2][0], H[0][1] + H[1][0]};
        double dC[6][6];
        dC_dtheta(e, nx, ny, layer_of_ez, layer_mat, elem_mat, layer_angle, theta, psi_x, matC, dC);
        double v = 0;
        for (int I = 0; I < 6; ++I)
            for (int K = 0; K < 6; ++K) v += wv[I] * dC[I][K] * eps[K];
        dJdth[e] = v;
    }
}

// grad[e] = - sum_q w_q |J_q| eps(lambda)_q^T (dC_e/dtheta_e) eps(u)_q.  One thread per element.
__global__ void k_adjoint_contract(int64_t n_elem, int nx, int ny, int NX, int NY, const double *__restrict__ geo,
                                   const int *__restrict__ layer_of_ez, const int *__restrict__ layer_mat,
                                   const int *__restrict__ elem_mat, const double *__restrict__ layer_angle,
                                   const double *__restrict__ theta, const double *__restrict__ psi_x,
                                   const double *__restrict__ matC,
                                   const double *__restrict__ u, const double *__restrict__ lam,
                                   double *__restrict__ grad) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n_elem) return;
    int ex = (int)(e % nx), ey = (int)((e / nx) % ny), ez = (int)(e / ((int64_t)nx * ny));
    double dC[6][6];
    dC_dtheta(e, nx, ny, layer_of_ez, layer_mat, elem_mat, layer_angle, theta, psi_x, matC, dC);
    double maxd = 0;
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) maxd = fmax(maxd, fabs(dC[i][j]));
    if (maxd == 0.0) {   // isotropic material: C does not depend on theta
        grad[e] = 0.0;
        return;
    }
    double ue[81], le[81];
    for (int a = 0; a < 27; ++a) {
        int64_t n = node_of(ex, ey, ez, a, NX, NY);
        for (int c = 0; c < 3; ++c) {
            ue[3 * a + c] = u[3 * n + c];
            le[3 * a + c] = lam[3 * n + c];
        }
    }
    double acc = 0.0;
    for (int q = 0; q < 27; ++q) {
        int qx = q % 3, qy = (q / 3) % 3, qz = q / 9;
        double gx = q2_gauss_pt(qx), gy = q2_gauss_pt(qy), gz = q2_gauss_pt(qz);
        const double *g = geo + 10 * (e * 27 + q);
        double Hu[3][3] = {{0}}, Hl[3][3] = {{0}};
        for (int a = 0; a < 27; ++a) {
            int i = a % 3, j = (a / 3) % 3, k = a / 9;
            double r0 = q2_dN(i, gx) * q2_N(j, gy) * q2_N(k, gz);
            double r1 = q2_N(i, gx) * q2_dN(j, gy) * q2_N(k, gz);
            double r2 = q2_N(i, gx) * q2_N(j, gy) * q2_dN(k, gz);
            double d[3];
            for (int c = 0; c < 3; ++c) d[c] = r0 * g[0 + c] + r1 * g[3 + c] + r2 * g[6 + c];
            for (int c = 0; c < 3; ++c)
                for (int dd = 0; dd < 3; ++dd) {
                    Hu[c][dd] += ue[3 * a + c] * d[dd];
                    Hl[c][dd] += le[3 * a + c] * d[dd];
                }
        }
        double eu[6] = {Hu[0][0], Hu[1][1], Hu[2][2], Hu[1][2] + Hu[2][1], Hu[0][2] + Hu[2][0], Hu[0][1] + Hu[1][0]};
        double el[6] = {Hl[0][0], Hl[1][1], Hl[2][2], Hl[1][2] + Hl[2][1], Hl[0][2] + Hl[2][0], Hl[0][1] + Hl[1][0]};
        double v = 0;
        for (int I = 0; I < 6; ++I)
            for (int K = 0; K < 6; ++K) v += el[I] * dC[I][K] * eu[K];
        acc += g[9] * v;
    }
    grad[e] = -acc;
}

void launch_stress_vjp(const MeshHost &m, const double *X, const double *C, const double *psi_x,
                       const int *layer_of_ez, const int *layer_mat, const int *elem_mat, const double *layer_angle,
                       const double *theta, const double *matC, const double *u, const double *w33, const double *w13,
                       double *dJdu, double *dJdth, cudaStream_t s) {
    k_stress_vjp<<<(unsigned)((m.n_elem + 127) / 128), 128, 0, s>>>(m.n_elem, m.nx, m.ny, m.NX, m.NY, X, C, psi_x,
                                                                   layer_of_ez, layer_mat, elem_mat, layer_angle,
                                                                   theta, matC, u, w33, w13, dJdu, dJdth);
    GL_CUDA(cudaGetLastError());
}

void launch_adjoint_contract(const MeshHost &m, const double *geo, const int *layer_of_ez, const int *layer_mat,
                             const int *elem_mat, const double *layer_angle, const double *theta, const double *psi_x,
                             const double *matC, const double *u, const double *lam, double *grad, cudaStream_t s) {
    k_adjoint_contract<<<(unsigned)((m.n_elem + 63) / 64), 64, 0, s>>>(m.n_elem, m.nx, m.ny, m.NX, m.NY, geo,
                                                                      layer_of_ez, layer_mat, elem_mat, layer_angle,
                                                                      theta, psi_x, matC, u, lam, grad);
    GL_CUDA(cudaGetLastError());
}

}  // namespace gl
