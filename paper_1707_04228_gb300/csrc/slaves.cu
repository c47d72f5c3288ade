// DOFs of the Q2 node grid that are not unknowns but fixed combinations of
// others ("slaves" of "masters"): the face and body centres of the 20-node
// serendipity element, and the last width plane under periodic width
// conditions.  Both constraints read u_Q2 = P u and wrap the Q2 kernels with a
// fill (slaves from masters) before and the transpose fold (masters += P^T y,
// slaves zeroed) after them.
//
// Serendipity (Section 2.1: the paper's own element) on the Q2 node grid.
//
// The serendipity space of an element is a subspace of its triquadratic Q2
// space, and its 20 nodes are the Q2 nodes with at most one odd local index
// (vertices and edge midpoints).  A serendipity field therefore is a Q2 field
// whose 7 other nodal values (face and body centres) are fixed combinations of
// the 20: u_Q2 = P u_20, with P the values of the 20 serendipity shape
// functions at the face and body centres:
//   face centre: -1/4 at the face's 4 corners, +1/2 at its 4 edge midpoints;
//   body centre: -1/4 at the 8 corners, +1/4 at the 12 edge midpoints.
// A face centre depends only on its face's nodes, so the same rule holds on
// the global grid: nodes with two or three odd indices ("slaves") take those
// combinations of their neighbours.  With the slaves' coordinates placed the
// same way the Q2 geometry map equals the serendipity map, and
//     K_20 = P^T K_Q2 P,  f_20 = P^T f_Q2,  sigma_20(u) = sigma_Q2(P u),
// all exactly (the 3x3x3 Gauss rule is the same).  The library keeps the Q2
// node numbering, treats the slave DOFs as eliminated (zero in the solver),
// and wraps the Q2 kernels: fill (u <- P u on the slave entries) before and
// the transpose fold (masters += P^T y, slaves zeroed) after them.
#include <algorithm>

#include "slaves.h"

namespace gl {

namespace {

// Masters of a global slave node (ix, iy, iz): count and (node, weight) pairs.
__device__ __forceinline__ int slave_stencil(int ix, int iy, int iz, int NX, int NY, int64_t *mn, double *mw) {
    const int o[3] = {ix & 1, iy & 1, iz & 1};
    const int nodd = o[0] + o[1] + o[2];
    if (nodd < 2) return 0;
    int cnt = 0;
    // offsets in {-1, 0, 1} along the odd axes (0 along an even axis)
    for (int dz = -o[2]; dz <= o[2]; ++dz)
        for (int dy = -o[1]; dy <= o[1]; ++dy)
            for (int dx = -o[0]; dx <= o[0]; ++dx) {
                const int moved = (dx != 0) + (dy != 0) + (dz != 0);
                const int still_odd = nodd - moved;   // odd indices left at the neighbour
                if (still_odd > 1) continue;          // the slave itself, or another slave
                double w;
                if (nodd == 3) w = still_odd == 0 ? -0.25 : 0.25;
                else w = still_odd == 0 ? -0.25 : 0.5;
                mn[cnt] = (int64_t)(ix + dx) + (int64_t)NX * ((iy + dy) + (int64_t)NY * (iz + dz));
                mw[cnt] = w;
                ++cnt;
            }
    return cnt;
}

__global__ void k_s20_fill(int NX, int NY, int NZ, double *__restrict__ v) {
    const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (n >= (int64_t)NX * NY * NZ) return;
    const int ix = (int)(n % NX), iy = (int)((n / NX) % NY), iz = (int)(n / ((int64_t)NX * NY));
    int64_t mn[20];
    double mw[20];
    const int cnt = slave_stencil(ix, iy, iz, NX, NY, mn, mw);
    if (!cnt) return;
    double s[3] = {0.0, 0.0, 0.0};
    for (int k = 0; k < cnt; ++k)
        for (int c = 0; c < 3; ++c) s[c] += mw[k] * v[3 * mn[k] + c];
    for (int c = 0; c < 3; ++c) v[3 * n + c] = s[c];
}

__global__ void k_s20_fold(int NX, int NY, int NZ, double *__restrict__ y) {
    const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (n >= (int64_t)NX * NY * NZ) return;
    const int ix = (int)(n % NX), iy = (int)((n / NX) % NY), iz = (int)(n / ((int64_t)NX * NY));
    int64_t mn[20];
    double mw[20];
    const int cnt = slave_stencil(ix, iy, iz, NX, NY, mn, mw);
    if (!cnt) return;
    double ys[3];
    for (int c = 0; c < 3; ++c) {
        ys[c] = y[3 * n + c];
        y[3 * n + c] = 0.0;
    }
    for (int k = 0; k < cnt; ++k)
        for (int c = 0; c < 3; ++c) atomicAdd(y + 3 * mn[k] + c, mw[k] * ys[c]);
}

}  // namespace

void s20_fill(const MeshHost &m, double *v, cudaStream_t s) {
    k_s20_fill<<<(unsigned)((m.n_nodes + 255) / 256), 256, 0, s>>>(m.NX, m.NY, m.NZ, v);
    GL_CUDA(cudaGetLastError());
}

void s20_fold(const MeshHost &m, double *y, cudaStream_t s) {
    k_s20_fold<<<(unsigned)((m.n_nodes + 255) / 256), 256, 0, s>>>(m.NX, m.NY, m.NZ, y);
    GL_CUDA(cudaGetLastError());
}

// Periodic width conditions (Section 3, the 39-ply study: u(s, 0, r) =
// u(s, W, r)): every node of the last width plane iy = NY - 1 is the slave
// of its partner on the first plane iy = 0 (weight 1).  Only the unknowns are
// identified; the nodes keep their own coordinates.
__global__ void k_per_fill(int NX, int NY, int NZ, double *__restrict__ v) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)NX * NZ) return;
    const int ix = (int)(t % NX), iz = (int)(t / NX);
    const int64_t master = ix + (int64_t)NX * ((int64_t)NY * iz);
    const int64_t slave = ix + (int64_t)NX * ((NY - 1) + (int64_t)NY * iz);
    for (int c = 0; c < 3; ++c) v[3 * slave + c] = v[3 * master + c];
}

__global__ void k_per_fold(int NX, int NY, int NZ, double *__restrict__ y) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)NX * NZ) return;
    const int ix = (int)(t % NX), iz = (int)(t / NX);
    const int64_t master = ix + (int64_t)NX * ((int64_t)NY * iz);
    const int64_t slave = ix + (int64_t)NX * ((NY - 1) + (int64_t)NY * iz);
    for (int c = 0; c < 3; ++c) {
        y[3 * master + c] += y[3 * slave + c];
        y[3 * slave + c] = 0.0;
    }
}

void slave_fill(const MeshHost &m, double *v, cudaStream_t s) {
    if (m.element == 1) s20_fill(m, v, s);
    if (m.periodic) {
        const int64_t n = (int64_t)m.NX * m.NZ;
        k_per_fill<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(m.NX, m.NY, m.NZ, v);
        GL_CUDA(cudaGetLastError());
    }
}

void slave_fold(const MeshHost &m, double *y, cudaStream_t s) {
    if (m.periodic) {
        const int64_t n = (int64_t)m.NX * m.NZ;
        k_per_fold<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(m.NX, m.NY, m.NZ, y);
        GL_CUDA(cudaGetLastError());
    }
    if (m.element == 1) s20_fold(m, y, s);
}

std::vector<int64_t> slave_dofs(const MeshHost &m) {
    std::vector<int64_t> out;
    if (m.element == 1) out = s20_slave_dofs(m);
    if (m.periodic)
        for (int iz = 0; iz < m.NZ; ++iz)
            for (int ix = 0; ix < m.NX; ++ix) {
                const int64_t n = ix + (int64_t)m.NX * ((m.NY - 1) + (int64_t)m.NY * iz);
                for (int c = 0; c < 3; ++c) out.push_back(3 * n + c);
            }
    std::sort(out.begin(), out.end());
    out.erase(std::unique(out.begin(), out.end()), out.end());
    return out;
}

std::vector<int64_t> s20_slave_dofs(const MeshHost &m) {
    std::vector<int64_t> out;
    for (int iz = 0; iz < m.NZ; ++iz)
        for (int iy = 0; iy < m.NY; ++iy)
            for (int ix = 0; ix < m.NX; ++ix)
                if ((ix & 1) + (iy & 1) + (iz & 1) >= 2) {
                    const int64_t n = (int64_t)ix + (int64_t)m.NX * (iy + (int64_t)m.NY * iz);
                    for (int c = 0; c < 3; ++c) out.push_back(3 * n + c);
                }
    return out;
}

}  // namespace gl
