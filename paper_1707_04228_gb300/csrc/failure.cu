// Quadratic damage-onset criterion of Section 3.2 (Eq. eq-Camanho):
//   F = sqrt((sigma_r^+ / s33)^2 + (tau_rs / s13)^2 + (tau_rl / s13)^2),
// sigma_r^+ = max(sigma_rr, 0), applied in the isotropic resin interfaces only
// (zero elsewhere), with the stresses recovered at the element centre and
// rotated into the local (s, l, r) frame.  One thread per element; the peak and
// its element come from a block reduction and a 64-bit atomic max on the
// (F, element) pair packed so that larger F wins.
#include "gl_internal.h"
#include "q2.cuh"

namespace gl {

namespace {

__device__ __forceinline__ int64_t fnode(int ex, int ey, int ez, int a, int NX, int NY) {
    return (int64_t)(2 * ex + a % 3) + (int64_t)NX * ((2 * ey + (a / 3) % 3) + (int64_t)NY * (2 * ez + a / 9));
}

}  // namespace

__global__ void __launch_bounds__(128) k_failure(int64_t n_elem, int nx, int ny, int NX, int NY,
                                                 const double *__restrict__ X, const double *__restrict__ C,
                                                 const double *__restrict__ psi_x, const uint8_t *__restrict__ resin,
                                                 const double *__restrict__ u, double s33a, double s13a,
                                                 double *__restrict__ F, unsigned long long *__restrict__ best) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    double fval = 0.0;
    if (e < n_elem && resin[e]) {
        const int ex = (int)(e % nx), ey = (int)((e / nx) % ny), ez = (int)(e / ((int64_t)nx * ny));
        double J[3][3] = {{0}}, G[3][3] = {{0}};
        for (int a = 0; a < 27; ++a) {
            const int i = a % 3, j = (a / 3) % 3, k = a / 9;
            const double d[3] = {q2_dN(i, 0.0) * q2_N(j, 0.0) * q2_N(k, 0.0), q2_N(i, 0.0) * q2_dN(j, 0.0) * q2_N(k, 0.0),
                                 q2_N(i, 0.0) * q2_N(j, 0.0) * q2_dN(k, 0.0)};
            if (d[0] == 0.0 && d[1] == 0.0 && d[2] == 0.0) continue;
            const int64_t nd = fnode(ex, ey, ez, a, NX, NY);
            for (int r = 0; r < 3; ++r)
                for (int c = 0; c < 3; ++c) {
                    J[r][c] += X[3 * nd + r] * d[c];
                    G[r][c] += u[3 * nd + r] * d[c];
                }
        }
        const double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                           J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                           J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
        const double id = 1.0 / det;
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
        double H[3][3];
        for (int c = 0; c < 3; ++c)
            for (int d = 0; d < 3; ++d) H[c][d] = G[c][0] * Ji[0][d] + G[c][1] * Ji[1][d] + G[c][2] * Ji[2][d];
        const double eps[6] = {H[0][0], H[1][1], H[2][2], H[1][2] + H[2][1], H[0][2] + H[2][0], H[0][1] + H[1][0]};
        const double *Ce = C + 36 * e;
        double sv[6];
        for (int i = 0; i < 6; ++i) {
            double v = 0;
            for (int j = 0; j < 6; ++j) v += Ce[6 * i + j] * eps[j];
            sv[i] = v;
        }
        const double S[3][3] = {{sv[0], sv[5], sv[4]}, {sv[5], sv[1], sv[3]}, {sv[4], sv[3], sv[2]}};
        double Rf[3][3];
        rot_width(psi_x[ex], Rf);
        // local (s, l, r) components: rr, rs, rl
        double srr = 0, srs = 0, srl = 0;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                srr += Rf[i][2] * S[i][j] * Rf[j][2];
                srs += Rf[i][0] * S[i][j] * Rf[j][2];
                srl += Rf[i][1] * S[i][j] * Rf[j][2];
            }
        const double a = fmax(srr, 0.0) / s33a, b = srs / s13a, c = srl / s13a;
        fval = sqrt(a * a + b * b + c * c);
    }
    if (e < n_elem) F[e] = fval;
    // block max of (F, element), then one atomic per block
    __shared__ double bf[128];
    __shared__ long long be[128];
    bf[threadIdx.x] = e < n_elem ? fval : -1.0;
    be[threadIdx.x] = e;
    __syncthreads();
    for (int o = 64; o > 0; o >>= 1) {
        if (threadIdx.x < o && bf[threadIdx.x + o] > bf[threadIdx.x]) {
            bf[threadIdx.x] = bf[threadIdx.x + o];
            be[threadIdx.x] = be[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0 && bf[0] >= 0.0) {
        // F >= 0: its bit pattern orders like the value; keep 40 bits of it and 24 of the element id
        unsigned long long key = ((unsigned long long)__double_as_longlong(bf[0]) >> 24) << 24;
        key |= (unsigned long long)(be[0] & 0xFFFFFF);
        atomicMax(best, key);
    }
}

void launch_failure(const MeshHost &m, const double *X, const double *C, const double *psi_x, const uint8_t *resin,
                    const double *u, double s33a, double s13a, double *F, unsigned long long *best, cudaStream_t s) {
    GL_CUDA(cudaMemsetAsync(best, 0, sizeof(unsigned long long), s));
    k_failure<<<(unsigned)((m.n_elem + 127) / 128), 128, 0, s>>>(m.n_elem, m.nx, m.ny, m.NX, m.NY, X, C, psi_x,
                                                                resin, u, s33a, s13a, F, best);
    GL_CUDA(cudaGetLastError());
}

}  // namespace gl
