// A set of independent laminates ("parts") solved together: their global
// vectors are concatenated (dof_off), their element data too (elem_off), and
// all their overlapping subdomains form one list, so every batched kernel of
// the factorisation, the GenEO setup and the PCG sweeps covers all parts in
// one launch.  A single laminate is a problem with one part.
#pragma once

#include <functional>

#include "factor.h"
#include "geneo.h"

namespace gl {

struct Part {
    const MeshHost *m = nullptr;
    std::vector<uint8_t> is_dir;   // part-local DOF mask of prescribed DOFs
    int64_t dof_off = 0, elem_off = 0;
    int sub0 = 0, sub1 = 0;        // its subdomains in the problem's list
};

struct Problem {
    std::vector<Part> parts;
    std::vector<SubBox> boxes;     // all subdomains
    std::vector<int> sub_part;     // owning part of each subdomain
    int64_t n_dof = 0, n_elem = 0;
    const double *C = nullptr, *geo = nullptr;   // element data indexed by global element id
    cudaStream_t stream = 0;
    int *d_err = nullptr;
    std::function<void(const char *)> stamp = [](const char *) {};
};

// Near-equal element boxes of one part grown by `overlap` (subdomain order z, y, x).
void part_boxes(const MeshHost &m, int px, int py, int pz, int overlap, std::vector<SubBox> &out);

// Symbolic factorisation of every subdomain (Dirichlet or Neumann matrix),
// with global DOF numbers and global element ids.
void problem_symbolic(const Problem &P, bool neumann, int leaf_nodes, std::vector<SubSymbolic> &syms);

// Element -> local index maps of the subdomains s0 .. s1-1 laid out by `plan`.
void problem_local_elems(const Problem &P, int s0, int s1, const FactorPlan &plan, LocalElems &E);

// GenEO coarse space of the whole problem: Neumann plan, coarse basis Z
// (Neumann-local layout, nev columns), kept eigenvalues, and the inverses of
// the per-part coarse matrices K_0 = Z^T K Z (block diagonal over parts).
struct Coarse {
    int nev = 0, n0 = 0, eig_iters = 0;
    int n_groups = 0;              // subdomain groups of the eigensolver
    int n_dropped = 0;             // coarse columns left out as linearly dependent (all parts)
    std::vector<int> part_dropped;  // the same per part
    FactorPlan PN;
    DBuf<double> Z, Kinv;
    std::vector<double> eig;
    std::vector<int64_t> koff;
    std::vector<int> kvoff, kn;
    DBuf<int64_t> d_koff;
    DBuf<int> d_kvoff, d_kn;
};

void problem_coarse(const Problem &P, const gl_opts &o, const FactorPlan &PD, int leaf_nodes, Coarse &out);

// z += Z K_0^{-1} Z^T r (per part blocks); c1, c2 scratch of n0 entries.
void coarse_apply(const Coarse &Cs, const double *r, double *z, double *c1, double *c2, cudaStream_t s);

}  // namespace gl
