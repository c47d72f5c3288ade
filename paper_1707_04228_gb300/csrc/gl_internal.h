// Internal declarations of the GenEO laminate library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "../../include/geneo_lam.h"

namespace gl {

struct Error {
    int code;
    std::string msg;
};

[[noreturn]] void fail(int code, const std::string &msg);

// A failed runtime call also leaves its error recorded as the thread's last
// error; it is read back (cleared) before failing, so that a recoverable error
// such as an allocation failure does not resurface at the next
// cudaGetLastError() of a later call.
#define GL_CUDA(x)                                                                   \
    do {                                                                             \
        cudaError_t e_ = (x);                                                        \
        if (e_ != cudaSuccess) {                                                     \
            cudaGetLastError();                                                      \
            ::gl::fail(e_ == cudaErrorMemoryAllocation ? GL_ERR_OOM : GL_ERR_CUDA,   \
                       std::string(#x) + ": " + cudaGetErrorString(e_));             \
        }                                                                            \
    } while (0)

#define GL_REQUIRE(cond, msg)                                                        \
    do {                                                                             \
        if (!(cond)) ::gl::fail(GL_ERR_INVALID_ARG, msg);                            \
    } while (0)

// Owning device buffer (cudaMalloc / cudaFree).
template <class T>
struct DBuf {
    T *p = nullptr;
    size_t n = 0;
    DBuf() = default;
    DBuf(const DBuf &) = delete;
    DBuf &operator=(const DBuf &) = delete;
    DBuf(DBuf &&o) noexcept : p(o.p), n(o.n) {
        o.p = nullptr;
        o.n = 0;
    }
    DBuf &operator=(DBuf &&o) noexcept {
        if (this != &o) {
            release();
            p = o.p;
            n = o.n;
            o.p = nullptr;
            o.n = 0;
        }
        return *this;
    }
    ~DBuf() { release(); }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
    }
    void alloc(size_t count) {
        release();
        if (count == 0) return;
        GL_CUDA(cudaMalloc(&p, count * sizeof(T)));
        n = count;
    }
    void upload(const std::vector<T> &h, cudaStream_t s) {
        alloc(h.size());
        if (n) GL_CUDA(cudaMemcpyAsync(p, h.data(), n * sizeof(T), cudaMemcpyHostToDevice, s));
    }
    void zero(cudaStream_t s) {
        if (n) GL_CUDA(cudaMemsetAsync(p, 0, n * sizeof(T), s));
    }
    T *get() const { return p; }
};

// Copies `count` elements from a host or device pointer into a host vector.
template <class T>
std::vector<T> fetch(const T *src, size_t count) {
    std::vector<T> out(count);
    if (count) GL_CUDA(cudaMemcpy(out.data(), src, count * sizeof(T), cudaMemcpyDefault));
    return out;
}

bool is_device_ptr(const void *p);

// ---------------------------------------------------------------- mesh
struct MeshHost {
    int nx = 0, ny = 0, nz = 0, NX = 0, NY = 0, NZ = 0;
    int64_t n_nodes = 0, n_dof = 0, n_elem = 0;
    int geometry = 0;
    int element = 0;                         // 0 Q2 (27 nodes), 1 serendipity (20 nodes; slaves.h)
    bool periodic = false;                   // periodic width: plane iy = NY-1 identified with iy = 0 (slaves.h)
    double R_inner = 0, limb_L = 0, arc_rad = 0;
    std::vector<double> sv, lv, rv;          // vertex coordinates (rv = depth from inner face)
    std::vector<double> tn, ln, rn;          // Q2 node parameters
    std::vector<int> layer_of_ez;            // layer of element row ez
    std::vector<int> layer_mat;
    std::vector<double> layer_angle;         // rad
    std::vector<double> theta;               // per element (rad), may be empty
    std::vector<double> node_dr;             // per node through-thickness offset (mm), may be empty
    std::vector<int> elem_mat;               // per element material overriding the layer's, may be empty
};

// ---------------------------------------------------------------- decomposition / symbolic
struct Supernode {
    int first;        // first local index (elimination order) of its pivots
    int p;            // pivots
    int q;            // structure rows below
    int depth;        // depth in the nested-dissection tree (root 0)
    int parent;       // index within the subdomain, -1 for the root
    int child[2];     // children (-1 if none)
    int64_t l_off;    // offset of its f x p column-major panel in the factor array
    int64_t row_off;  // offset of its f local row indices in the row array
    int64_t emap_off; // offset of (element, 81 front positions) list
    int n_elem_pairs; // number of elements assembling into its front
    int64_t rel_off;  // offset of its q-entry relative map into the parent front
    int box[6];       // node box of its subtree region (x0,x1,y0,y1,z0,z1) inclusive
};

struct SubSymbolic {
    int n = 0;                          // local DOFs
    std::vector<int64_t> gdof;          // local (elimination order) -> global DOF
    std::vector<Supernode> sn;          // postorder
    std::vector<int> rows;              // concatenated front rows (local indices)
    std::vector<int> rel;               // concatenated child -> parent front positions
    std::vector<int> pair_elem;         // concatenated element ids of (front, element) pairs
    std::vector<int16_t> pair_pos;      // 81 front positions per pair (-1: skip)
    int64_t l_size = 0;                 // factor entries
    int max_depth = 0;
};

struct SubBox {
    int ebox[6];     // element box [x0,x1) [y0,y1) [z0,z1) (overlapped)
    int nbox[6];     // node box inclusive
    bool art[6];     // face is artificial (interior to the global domain)
};

void build_symbolic(const MeshHost &m, const SubBox &b, const std::vector<uint8_t> &dof_is_dir,
                    bool neumann, int leaf_nodes, SubSymbolic &out);

// ---------------------------------------------------------------- kernels (launchers)
void launch_node_coords(const MeshHost &m, const double *tn, const double *ln, const double *rn,
                        const double *dr, double *X, cudaStream_t s);
void launch_elem_material(int64_t n_elem, int nx, int ny, const int *layer_of_ez, const int *layer_mat,
                          const int *elem_mat, const double *layer_angle, const double *theta, const double *psi,
                          const double *matC, double *C, cudaStream_t s);
void launch_elem_geometry(const MeshHost &m, const double *X, double *geo, cudaStream_t s);
void launch_traction(const MeshHost &m, const double *X, int face, const double t[3], double *f,
                     cudaStream_t s);
void launch_ku(const MeshHost &m, const double *C, const double *geo, const double *x, double *y,
               cudaStream_t s);
void launch_stress(const MeshHost &m, const double *X, const double *C, const double *psi,
                   const double *u, double *s33, double *t13, cudaStream_t s);
void launch_failure(const MeshHost &m, const double *X, const double *C, const double *psi_x, const uint8_t *resin,
                    const double *u, double s33a, double s13a, double *F, unsigned long long *best, cudaStream_t s);
// FP64 FMA probe on the current device (probe.cu): flops per second.
double fp64_probe(int iters, int reps, int *n_sm, double *ms_out);
// Fails with GL_ERR_INVALID_ARG unless [p, p + bytes) lies inside one device
// allocation (cuMemGetAddressRange; no allocation is made).
void require_device_span(const void *p, size_t bytes, const char *what);
// Stress recovery into caller device buffers with the resin peak reduced
// through a fixed file-scope device scratch (no device allocation).
void stress_noalloc(const MeshHost &m, int device, const double *X, const double *C, const double *psi_x,
                    const uint8_t *resin, const double *u, double *s33, double *t13, double *peak, cudaStream_t s);
void launch_stress_vjp(const MeshHost &m, const double *X, const double *C, const double *psi_x,
                       const int *layer_of_ez, const int *layer_mat, const int *elem_mat, const double *layer_angle,
                       const double *theta, const double *matC, const double *u, const double *w33, const double *w13,
                       double *dJdu, double *dJdth, cudaStream_t s);
void launch_adjoint_contract(const MeshHost &m, const double *geo, const int *layer_of_ez, const int *layer_mat,
                             const int *elem_mat, const double *layer_angle, const double *theta, const double *psi_x,
                             const double *matC, const double *u, const double *lam, double *grad, cudaStream_t s);

}  // namespace gl
