// Q2 (triquadratic, 27-node) reference element on the device.
//
// 1D quadratic Lagrange basis on the nodes {-1, 0, 1} and the 3-point Gauss
// rule (full integration, Section 2.1).  Local node a = i + 3j + 9k sits at
// reference coordinates (i-1, j-1, k-1); Gauss point q = qx + 3qy + 9qz.
#pragma once

namespace gl {

__device__ __forceinline__ double q2_gauss_pt(int q) {
    // +-sqrt(3/5), 0
    return q == 1 ? 0.0 : (q == 0 ? -0.77459666924148337704 : 0.77459666924148337704);
}
__device__ __forceinline__ double q2_gauss_wt(int q) { return q == 1 ? 8.0 / 9.0 : 5.0 / 9.0; }

__device__ __forceinline__ double q2_N(int i, double x) {
    return i == 0 ? 0.5 * x * (x - 1.0) : (i == 1 ? 1.0 - x * x : 0.5 * x * (x + 1.0));
}
__device__ __forceinline__ double q2_dN(int i, double x) {
    return i == 0 ? x - 0.5 : (i == 1 ? -2.0 * x : x + 0.5);
}

// Tables at the Gauss points: N[q][i] = N_i(g_q), D[q][i] = N_i'(g_q).
struct Q2Tables {
    double N[3][3], D[3][3];
    __device__ __forceinline__ void init() {
#pragma unroll
        for (int q = 0; q < 3; ++q)
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                N[q][i] = q2_N(i, q2_gauss_pt(q));
                D[q][i] = q2_dN(i, q2_gauss_pt(q));
            }
    }
};

// Rotation about the width axis (l / y): maps e_s to (cos a, 0, -sin a).
__device__ __forceinline__ void rot_width(double a, double R[3][3]) {
    double c = cos(a), s = sin(a);
    R[0][0] = c;  R[0][1] = 0; R[0][2] = s;
    R[1][0] = 0;  R[1][1] = 1; R[1][2] = 0;
    R[2][0] = -s; R[2][1] = 0; R[2][2] = c;
}

}  // namespace gl
