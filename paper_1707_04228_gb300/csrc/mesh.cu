// Mesh, material and element-level setup kernels, loads and stress recovery.
//
// Geometry: structured Q2 node grid; the curved corner follows the map of
// Section 3 (x = L + r sin psi, y = l, z = r cos psi) with straight limbs
// appended along the tangent.  Materials: Table 1 constants rotated by
// R = R_l(psi + theta) R_r(phi) (ply angle phi about the normal, misalignment
// theta and the curved frame angle psi about the width axis), here through the
// 6x6 Bond matrix: C_global = M C_material M^T.
#include "gl_internal.h"
#include "q2.cuh"

namespace gl {

// ---------------------------------------------------------------- node coordinates

// dr (may be NULL): per-node offset of the through-thickness coordinate, the
// geometric wrinkle r^ = r + f(s, l, r) of Section 3, applied before the map.
__global__ void k_node_coords(int NX, int NY, int NZ, int geometry, double R_inner, double L,
                              double arc, const double *__restrict__ tn, const double *__restrict__ ln,
                              const double *__restrict__ rn, const double *__restrict__ dr,
                              double *__restrict__ X) {
    int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t total = (int64_t)NX * NY * NZ;
    if (n >= total) return;
    int ix = (int)(n % NX);
    int iy = (int)((n / NX) % NY);
    int iz = (int)(n / ((int64_t)NX * NY));
    double t = tn[ix], l = ln[iy], d = rn[iz] + (dr ? dr[n] : 0.0);
    double x, y = l, z;
    if (geometry == 0) {
        x = t;
        z = d;
    } else {
        double r = R_inner + d;
        double psi = fmin(fmax(t, 0.0), 1.0) * arc;
        double sp = sin(psi), cp = cos(psi);
        double ext = t < 0.0 ? t * L : (t > 1.0 ? (t - 1.0) * L : 0.0);
        x = L + r * sp + ext * cp;
        z = r * cp - ext * sp;
    }
    X[3 * n + 0] = x;
    X[3 * n + 1] = y;
    X[3 * n + 2] = z;
}

void launch_node_coords(const MeshHost &m, const double *tn, const double *ln, const double *rn,
                        const double *dr, double *X, cudaStream_t s) {
    int64_t n = m.n_nodes;
    k_node_coords<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(m.NX, m.NY, m.NZ, m.geometry, m.R_inner,
                                                             m.limb_L, m.arc_rad, tn, ln, rn, dr, X);
    GL_CUDA(cudaGetLastError());
}

// ---------------------------------------------------------------- element material

// Bond matrix M (stress rotation, Voigt 11,22,33,23,13,12) for a rotation a:
// sigma' = M sigma when sigma'_ij = a_ik a_jl sigma_kl.
__device__ void bond_matrix(const double a[3][3], double M[6][6]) {
    const int I0[6] = {0, 1, 2, 1, 0, 0}, I1[6] = {0, 1, 2, 2, 2, 1};
    for (int r = 0; r < 6; ++r) {
        int i = I0[r], j = I1[r];
        for (int c = 0; c < 6; ++c) {
            int k = I0[c], l = I1[c];
            // sigma'_ij = sum_kl a_ik a_jl sigma_kl; Voigt column c collects (k,l) and (l,k)
            double v = a[i][k] * a[j][l];
            if (k != l) v += a[i][l] * a[j][k];
            M[r][c] = v;
        }
    }
}

// elem_mat (may be NULL): per-element material index overriding the layer's.
__global__ void k_elem_material(int64_t n_elem, int nx, int ny, const int *__restrict__ layer_of_ez,
                                const int *__restrict__ layer_mat, const int *__restrict__ elem_mat,
                                const double *__restrict__ layer_angle,
                                const double *__restrict__ theta, const double *__restrict__ psi_x,
                                const double *__restrict__ matC, double *__restrict__ C) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n_elem) return;
    int ex = (int)(e % nx);
    int ez = (int)(e / ((int64_t)nx * ny));
    int layer = layer_of_ez[ez];
    int mat = elem_mat ? elem_mat[e] : layer_mat[layer];
    double phi = layer_angle[layer];
    double a = psi_x[ex] + (theta ? theta[e] : 0.0);
    double Ry[3][3];
    rot_width(a, Ry);
    double cp = cos(phi), sp = sin(phi);
    double Rz[3][3] = {{cp, -sp, 0}, {sp, cp, 0}, {0, 0, 1}};
    double R[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double v = 0;
            for (int k = 0; k < 3; ++k) v += Ry[i][k] * Rz[k][j];
            R[i][j] = v;
        }
    double M[6][6];
    bond_matrix(R, M);
    const double *Cm = matC + 36 * mat;
    double T[6][6];
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) {
            double v = 0;
            for (int k = 0; k < 6; ++k) v += M[i][k] * Cm[6 * k + j];
            T[i][j] = v;
        }
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) {
            double v = 0;
            for (int k = 0; k < 6; ++k) v += T[i][k] * M[j][k];
            C[36 * e + 6 * i + j] = v;
        }
}

void launch_elem_material(int64_t n_elem, int nx, int ny, const int *layer_of_ez, const int *layer_mat,
                          const int *elem_mat, const double *layer_angle, const double *theta, const double *psi_x,
                          const double *matC, double *C, cudaStream_t s) {
    k_elem_material<<<(unsigned)((n_elem + 127) / 128), 128, 0, s>>>(n_elem, nx, ny, layer_of_ez, layer_mat,
                                                                    elem_mat, layer_angle, theta, psi_x, matC, C);
    GL_CUDA(cudaGetLastError());
}

// ---------------------------------------------------------------- element geometry

__device__ __forceinline__ int64_t elem_node(int ex, int ey, int ez, int a, int NX, int NY) {
    int i = a % 3, j = (a / 3) % 3, k = a / 9;
    return (int64_t)(2 * ex + i) + (int64_t)NX * ((2 * ey + j) + (int64_t)NY * (2 * ez + k));
}

// geo[(e*27 + q)*10 + 0..8] = J^{-1} (row-major, dxi_i/dx_j), [9] = w_q det J.
__global__ void k_elem_geometry(int64_t n_elem, int nx, int ny, int NX, int NY, const double *__restrict__ X,
                                double *__restrict__ geo, int *__restrict__ bad) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n_elem * 27) return;
    int64_t e = t / 27;
    int q = (int)(t % 27);
    int ex = (int)(e % nx), ey = (int)((e / nx) % ny), ez = (int)(e / ((int64_t)nx * ny));
    int qx = q % 3, qy = (q / 3) % 3, qz = q / 9;
    double gx = q2_gauss_pt(qx), gy = q2_gauss_pt(qy), gz = q2_gauss_pt(qz);
    double J[3][3] = {{0}};
    for (int a = 0; a < 27; ++a) {
        int i = a % 3, j = (a / 3) % 3, k = a / 9;
        double d0 = q2_dN(i, gx) * q2_N(j, gy) * q2_N(k, gz);
        double d1 = q2_N(i, gx) * q2_dN(j, gy) * q2_N(k, gz);
        double d2 = q2_N(i, gx) * q2_N(j, gy) * q2_dN(k, gz);
        const double *x = X + 3 * elem_node(ex, ey, ez, a, NX, NY);
        for (int r = 0; r < 3; ++r) {
            J[r][0] += x[r] * d0;
            J[r][1] += x[r] * d1;
            J[r][2] += x[r] * d2;
        }
    }
    double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                 J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                 J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
    if (!(det > 0.0)) atomicExch(bad, 1);
    double id = 1.0 / det;
    double *g = geo + 10 * t;
    g[0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) * id;
    g[1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) * id;
    g[2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) * id;
    g[3] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) * id;
    g[4] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) * id;
    g[5] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) * id;
    g[6] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) * id;
    g[7] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) * id;
    g[8] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) * id;
    g[9] = q2_gauss_wt(qx) * q2_gauss_wt(qy) * q2_gauss_wt(qz) * det;
}

void launch_elem_geometry(const MeshHost &m, const double *X, double *geo, cudaStream_t s) {
    DBuf<int> bad;
    bad.alloc(1);
    bad.zero(s);
    int64_t n = m.n_elem * 27;
    k_elem_geometry<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(m.n_elem, m.nx, m.ny, m.NX, m.NY, X, geo,
                                                               bad.p);
    GL_CUDA(cudaGetLastError());
    int h = 0;
    GL_CUDA(cudaMemcpyAsync(&h, bad.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    GL_CUDA(cudaStreamSynchronize(s));
    if (h) fail(GL_ERR_INVALID_ARG, "mesh has an element with non-positive Jacobian determinant");
}

// ---------------------------------------------------------------- traction loads

__global__ void k_traction(int nx, int ny, int nz, int NX, int NY, int face, double t0, double t1, double t2,
                           const double *__restrict__ X, double *__restrict__ f) {
    int axis = face / 2, side = face % 2;
    int n1 = axis == 0 ? ny : nx, n2 = axis == 2 ? ny : nz;
    int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t nfe = (int64_t)n1 * n2;
    if (tid >= nfe * 9) return;
    int64_t fe = tid / 9;
    int gq = (int)(tid % 9);
    int u = (int)(fe % n1), v = (int)(fe / n1);
    int ex, ey, ez;
    int nfix = axis == 0 ? nx : (axis == 1 ? ny : nz);
    int efix = side == 0 ? 0 : nfix - 1;
    if (axis == 0) { ex = efix; ey = u; ez = v; }
    else if (axis == 1) { ex = u; ey = efix; ez = v; }
    else { ex = u; ey = v; ez = efix; }
    int o1 = axis == 0 ? 1 : 0, o2 = axis == 2 ? 1 : 2;
    double xi[3];
    xi[axis] = side == 0 ? -1.0 : 1.0;
    xi[o1] = q2_gauss_pt(gq % 3);
    xi[o2] = q2_gauss_pt(gq / 3);
    double w = q2_gauss_wt(gq % 3) * q2_gauss_wt(gq / 3);
    double J[3][3] = {{0}};
    double Nv[27];
    for (int a = 0; a < 27; ++a) {
        int i = a % 3, j = (a / 3) % 3, k = a / 9;
        double n0 = q2_N(i, xi[0]), n1v = q2_N(j, xi[1]), n2v = q2_N(k, xi[2]);
        double d[3] = {q2_dN(i, xi[0]) * n1v * n2v, n0 * q2_dN(j, xi[1]) * n2v, n0 * n1v * q2_dN(k, xi[2])};
        Nv[a] = n0 * n1v * n2v;
        const double *x = X + 3 * elem_node(ex, ey, ez, a, NX, NY);
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) J[r][c] += x[r] * d[c];
    }
    double cx = J[1][o1] * J[2][o2] - J[2][o1] * J[1][o2];
    double cy = J[2][o1] * J[0][o2] - J[0][o1] * J[2][o2];
    double cz = J[0][o1] * J[1][o2] - J[1][o1] * J[0][o2];
    double dA = sqrt(cx * cx + cy * cy + cz * cz) * w;
    for (int a = 0; a < 27; ++a) {
        if (Nv[a] == 0.0) continue;
        int64_t n = elem_node(ex, ey, ez, a, NX, NY);
        double s = Nv[a] * dA;
        atomicAdd(f + 3 * n + 0, s * t0);
        atomicAdd(f + 3 * n + 1, s * t1);
        atomicAdd(f + 3 * n + 2, s * t2);
    }
}

void launch_traction(const MeshHost &m, const double *X, int face, const double t[3], double *f, cudaStream_t s) {
    int axis = face / 2;
    int64_t n1 = axis == 0 ? m.ny : m.nx, n2 = axis == 2 ? m.ny : m.nz;
    int64_t n = n1 * n2 * 9;
    k_traction<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(m.nx, m.ny, m.nz, m.NX, m.NY, face, t[0], t[1], t[2],
                                                          X, f);
    GL_CUDA(cudaGetLastError());
}

// ---------------------------------------------------------------- stress recovery

// sigma = C_e eps(u) at the element centre, rotated into the local (s, l, r)
// frame: sigma_loc = Rf^T sigma Rf with Rf = R_l(psi); s33 = sigma_rr, t13 = tau_rs.
__global__ void k_stress(int64_t n_elem, int nx, int ny, int NX, int NY, const double *__restrict__ X,
                         const double *__restrict__ C, const double *__restrict__ psi_x,
                         const double *__restrict__ u, double *__restrict__ s33, double *__restrict__ t13) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n_elem) return;
    int ex = (int)(e % nx), ey = (int)((e / nx) % ny), ez = (int)(e / ((int64_t)nx * ny));
    double J[3][3] = {{0}}, G[3][3] = {{0}};   // G[c][d] = du_c/dxi_d
    for (int a = 0; a < 27; ++a) {
        int i = a % 3, j = (a / 3) % 3, k = a / 9;
        double d[3] = {q2_dN(i, 0.0) * q2_N(j, 0.0) * q2_N(k, 0.0), q2_N(i, 0.0) * q2_dN(j, 0.0) * q2_N(k, 0.0),
                       q2_N(i, 0.0) * q2_N(j, 0.0) * q2_dN(k, 0.0)};
        if (d[0] == 0.0 && d[1] == 0.0 && d[2] == 0.0) continue;
        int64_t n = elem_node(ex, ey, ez, a, NX, NY);
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) {
                J[r][c] += X[3 * n + r] * d[c];
                G[r][c] += u[3 * n + r] * d[c];
            }
    }
    double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                 J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                 J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
    double id = 1.0 / det;
    double Ji[3][3];
    Ji[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) * id;
    Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) * id;
    Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) * id;
    Ji[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) * id;
    Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) * id;
    Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) * id;
    Ji[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) * id;
    Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) * id;
    Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) * id;
    double H[3][3];   // du_c/dx_d
    for (int c = 0; c < 3; ++c)
        for (int d = 0; d < 3; ++d) H[c][d] = G[c][0] * Ji[0][d] + G[c][1] * Ji[1][d] + G[c][2] * Ji[2][d];
    double eps[6] = {H[0][0], H[1][1], H[2][2], H[1][2] + H[2][1], H[0][2] + H[2][0], H[0][1] + H[1][0]};
    const double *Ce = C + 36 * e;
    double sv[6];
    for (int i = 0; i < 6; ++i) {
        double v = 0;
        for (int j = 0; j < 6; ++j) v += Ce[6 * i + j] * eps[j];
        sv[i] = v;
    }
    double S[3][3] = {{sv[0], sv[5], sv[4]}, {sv[5], sv[1], sv[3]}, {sv[4], sv[3], sv[2]}};
    double Rf[3][3];
    rot_width(psi_x[ex], Rf);
    // sigma_loc[a][b] = sum_ij Rf[i][a] S[i][j] Rf[j][b]
    double l22 = 0, l02 = 0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            l22 += Rf[i][2] * S[i][j] * Rf[j][2];
            l02 += Rf[i][0] * S[i][j] * Rf[j][2];
        }
    if (s33) s33[e] = l22;
    if (t13) t13[e] = l02;
}

void launch_stress(const MeshHost &m, const double *X, const double *C, const double *psi_x, const double *u,
                   double *s33, double *t13, cudaStream_t s) {
    k_stress<<<(unsigned)((m.n_elem + 127) / 128), 128, 0, s>>>(m.n_elem, m.nx, m.ny, m.NX, m.NY, X, C, psi_x, u,
                                                               s33, t13);
    GL_CUDA(cudaGetLastError());
}

}  // namespace gl
