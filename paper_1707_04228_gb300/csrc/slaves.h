// DOFs of the Q2 grid fixed by constraints (slaves.cu): the face/body centres
// of the 20-node serendipity element (fixed combinations of the element's 20
// nodes) and the last width plane under periodic width conditions (equal to
// the first plane).
#pragma once

#include "gl_internal.h"

namespace gl {

// Weight of local node a in local slave node b of one element (local index
// i + 3j + 9k, i, j, k in {0, 1, 2}): the value of a's serendipity shape
// function at b; 0 if b is not a slave or a is not in its stencil.
//   face centre (two indices 1): -1/4 at the face's corners, +1/2 at its edge midpoints;
//   body centre (1, 1, 1):       -1/4 at the corners, +1/4 at the edge midpoints.
__device__ __forceinline__ double s20_weight(int b, int a) {
    const int bi = b % 3, bj = (b / 3) % 3, bk = b / 9;
    const int ai = a % 3, aj = (a / 3) % 3, ak = a / 9;
    const int bodd = (bi == 1) + (bj == 1) + (bk == 1);
    const int aodd = (ai == 1) + (aj == 1) + (ak == 1);
    if (bodd < 2 || aodd > 1) return 0.0;
    if (bodd == 3) return aodd == 0 ? -0.25 : 0.25;
    const int d = bi != 1 ? 0 : (bj != 1 ? 1 : 2);   // the face lies at the even index of b
    const int bd = d == 0 ? bi : (d == 1 ? bj : bk);
    const int ad = d == 0 ? ai : (d == 1 ? aj : ak);
    if (ad != bd) return 0.0;
    return aodd == 0 ? -0.25 : 0.5;
}

__device__ __forceinline__ bool s20_is_slave(int a) {
    return (a % 3 == 1) + ((a / 3) % 3 == 1) + (a / 9 == 1) >= 2;
}

// Global grid: v[slave] <- sum of weights x v[masters] (3 components per node).
void s20_fill(const MeshHost &m, double *v, cudaStream_t s);
// Transpose: y[master] += weight x y[slave] for every slave, then y[slave] = 0.
void s20_fold(const MeshHost &m, double *y, cudaStream_t s);
// DOFs of the slave nodes (eliminated from the serendipity system).
std::vector<int64_t> s20_slave_dofs(const MeshHost &m);

// Every constraint of the mesh (serendipity and/or periodic width), in the
// order that composes them: fill = periodic after serendipity, fold the
// reverse.  slave_dofs: all slave DOFs, sorted.
inline bool has_slaves(const MeshHost &m) { return m.element == 1 || m.periodic; }
void slave_fill(const MeshHost &m, double *v, cudaStream_t s);
void slave_fold(const MeshHost &m, double *y, cudaStream_t s);
std::vector<int64_t> slave_dofs(const MeshHost &m);

}  // namespace gl
