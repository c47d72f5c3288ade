// Matrix-free element-by-element K u for Q2 hexahedra in FP64 (Section 2.3:
// the iterative solver only needs products with the sparse stiffness K).
//
// y = sum_e P_e^T K_e P_e x with K_e = sum_q w_q |J_q| B_q^T C_e B_q (full
// 3x3x3 Gauss integration), never forming K_e: per element the 27x3 nodal
// values are gathered into shared memory, interpolated to the 27 Gauss points
// by three sum-factorised 1D contractions and differentiated there, the stress
// sigma = C_e eps is formed pointwise, and the transposed contractions give
// the 81 element residual entries, scatter-added with FP64 atomics.
//
// One 32-lane warp per element (27 active lanes: lane t is node t in the
// gather/scatter, Gauss point t in the pointwise stage); EPB elements per
// block.  The product is FP64-ALU bound on this part (5,346 FMA + 162 MUL per
// element against 2,448 B of element data and 16 B per DOF of vector traffic).
//
// The same element core serves the global product (node-major global
// vectors) and the subdomain-local products of the GenEO setup (local
// vectors reached through per-element index maps, optional diagonal
// scaling on both sides, several vectors per call).
#include "geneo.h"
#include "q2.cuh"
#include "slaves.h"

namespace gl {

constexpr int KU_EPB = 4;

struct KuSmem {
    double U[3][27], A[3][27], B[3][27], AA[3][27], AB[3][27], BA[3][27], C[36];
};

// Derivative of the Lagrange basis on the 3 Gauss points at the Gauss points:
// D[q][r] = l_r'(g_q), g = (-a, 0, a), a = sqrt(3/5).  A quadratic sampled at
// the Gauss points is differentiated there exactly by it (collocation).
struct GaussDeriv {
    double D[3][3];
    __device__ __forceinline__ void init() {
        const double a = sqrt(0.6), h = 0.5 / a;
        D[0][0] = -3.0 * h; D[0][1] = 4.0 * h;  D[0][2] = -h;
        D[1][0] = -h;       D[1][1] = 0.0;      D[1][2] = h;
        D[2][0] = h;        D[2][1] = -4.0 * h; D[2][2] = 3.0 * h;
    }
};

// Element residual of the values in s.U (component-major, node t = i + 3j + 9k).
// On return lane t (< 27) holds the three components of node t in out[].
// Collocation form of the sum factorisation: u is interpolated to the 27
// Gauss points by three 1D contractions with N[q][i], differentiated there
// along each axis with the Gauss-point derivative matrix (exact: u is
// quadratic along every line), and the flux goes back through the transposed
// steps -- 5,346 FMA + 162 MUL per element against 6,318 + 162 for
// derivatives taken from the nodes.
__device__ __forceinline__ void ku_core(KuSmem &s, const Q2Tables &T, const GaussDeriv &G, int t,
                                        const double *__restrict__ geo_e, double out[3]) {
    const bool on = t < 27;
    const int ti = t % 3, tj = (t / 3) % 3, tk = t / 9;
    // interpolation along x (lane = (qx, j, k)), y (lane = (qx, qy, k)), z (lane = Gauss point)
    if (on) {
        for (int c = 0; c < 3; ++c) {
            const double *u = &s.U[c][3 * tj + 9 * tk];
            s.A[c][t] = T.N[ti][0] * u[0] + T.N[ti][1] * u[1] + T.N[ti][2] * u[2];
        }
    }
    __syncwarp();
    if (on) {
        for (int c = 0; c < 3; ++c) {
            const double *a = &s.A[c][ti + 9 * tk];
            s.AA[c][t] = T.N[tj][0] * a[0] + T.N[tj][1] * a[3] + T.N[tj][2] * a[6];
        }
    }
    __syncwarp();
    if (on) {
        for (int c = 0; c < 3; ++c) {
            const double *a = &s.AA[c][ti + 3 * tj];
            s.B[c][t] = T.N[tk][0] * a[0] + T.N[tk][1] * a[9] + T.N[tk][2] * a[18];
        }
    }
    __syncwarp();
    // reference gradients at the Gauss point, pointwise stress and reference flux
    double F[3][3];
    if (on) {
        double Gr[3][3];
        for (int c = 0; c < 3; ++c) {
            const double *bx = &s.B[c][3 * tj + 9 * tk];
            const double *by = &s.B[c][ti + 9 * tk];
            const double *bz = &s.B[c][ti + 3 * tj];
            Gr[c][0] = G.D[ti][0] * bx[0] + G.D[ti][1] * bx[1] + G.D[ti][2] * bx[2];
            Gr[c][1] = G.D[tj][0] * by[0] + G.D[tj][1] * by[3] + G.D[tj][2] * by[6];
            Gr[c][2] = G.D[tk][0] * bz[0] + G.D[tk][1] * bz[9] + G.D[tk][2] * bz[18];
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
            for (int d = 0; d < 3; ++d) H[c][d] = Gr[c][0] * Ji[0 + d] + Gr[c][1] * Ji[3 + d] + Gr[c][2] * Ji[6 + d];
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
    // transposed derivatives (lane = Gauss point):
    //   V = sum_r D[r][qx] F0[r,qy,qz] + D[r][qy] F1[qx,r,qz] + D[r][qz] F2[qx,qy,r]
    if (on) {
        for (int c = 0; c < 3; ++c) {
            const double *f0 = &s.AA[c][3 * tj + 9 * tk];
            const double *f1 = &s.AB[c][ti + 9 * tk];
            const double *f2 = &s.BA[c][ti + 3 * tj];
            s.A[c][t] = G.D[0][ti] * f0[0] + G.D[1][ti] * f0[1] + G.D[2][ti] * f0[2] + G.D[0][tj] * f1[0] +
                        G.D[1][tj] * f1[3] + G.D[2][tj] * f1[6] + G.D[0][tk] * f2[0] + G.D[1][tk] * f2[9] +
                        G.D[2][tk] * f2[18];
        }
    }
    __syncwarp();
    // transposed interpolation along z (lane = (qx, qy, k)), y (lane = (qx, j, k)), x (lane = node)
    if (on) {
        for (int c = 0; c < 3; ++c) {
            const double *v = &s.A[c][ti + 3 * tj];
            s.U[c][t] = T.N[0][tk] * v[0] + T.N[1][tk] * v[9] + T.N[2][tk] * v[18];
        }
    }
    __syncwarp();
    if (on) {
        for (int c = 0; c < 3; ++c) {
            const double *v = &s.U[c][ti + 9 * tk];
            s.B[c][t] = T.N[0][tj] * v[0] + T.N[1][tj] * v[3] + T.N[2][tj] * v[6];
        }
    }
    __syncwarp();
    if (on) {
        for (int c = 0; c < 3; ++c) {
            const double *v = &s.B[c][3 * tj + 9 * tk];
            out[c] = T.N[0][ti] * v[0] + T.N[1][ti] * v[1] + T.N[2][ti] * v[2];
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
    GaussDeriv Gd;
    Gd.init();
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
    ku_core(s, T, Gd, t, geo + 270 * e, out);
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
    GaussDeriv Gd;
    Gd.init();
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
    ku_core(s, T, Gd, t, geo + 270 * eg, out);
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
                                                         double *__restrict__ y, int nv, int s20) {
    __shared__ KuSmem sm[KU_EPB];
    const int w = threadIdx.x >> 5, t = threadIdx.x & 31;
    const int64_t pi = (int64_t)blockIdx.x * KU_EPB + w;
    if (pi >= n_pairs) return;
    KuSmem &s = sm[w];
    Q2Tables T;
    T.init();
    GaussDeriv Gd;
    Gd.init();
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
        if (s20) {
            // serendipity: the 7 face/body-centre values from the element's 20 nodes
            double f[3] = {0.0, 0.0, 0.0};
            if (t < 27 && s20_is_slave(t))
                for (int a = 0; a < 27; ++a) {
                    const double w = s20_weight(t, a);
                    if (w != 0.0)
                        for (int c = 0; c < 3; ++c) f[c] += w * s.U[c][a];
                }
            __syncwarp();
            if (t < 27 && s20_is_slave(t))
                for (int c = 0; c < 3; ++c) s.U[c][t] = f[c];
            __syncwarp();
        }
        double out[3];
        ku_core(s, T, Gd, t, geo + 270 * e, out);
        if (s20) {
            // transpose: the slaves' residuals go to the 20 nodes
            if (t < 27)
                for (int c = 0; c < 3; ++c) s.A[c][t] = out[c];
            __syncwarp();
            if (t < 27 && !s20_is_slave(t))
                for (int b = 0; b < 27; ++b) {
                    const double w = s20_weight(b, t);
                    if (w != 0.0)
                        for (int c = 0; c < 3; ++c) out[c] += w * s.A[c][b];
                }
            __syncwarp();
        }
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
                                                   P.d_vec_len.p, C, geo, xi, x, y, nv, P.s20 ? 1 : 0);
    GL_CUDA(cudaGetLastError());
}

}  // namespace gl
