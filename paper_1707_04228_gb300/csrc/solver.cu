// Solver context, setup, PCG driver and the C ABI (include/geneo_lam.h).
//
// Section 2.3: CG on P K u = P f (Eq. eq-pre) with P the two-level additive
// overlapping Schwarz preconditioner
//     P = Z K_0^{-1} Z^T + sum_j R_j^T A_j^{-1} R_j,
// A_j the Dirichlet matrices of the overlapping subdomains (direct solves),
// Z the GenEO coarse basis (Xi_j-weighted low-energy eigenvectors of the local
// Neumann matrices, Fig. eig), K_0 = Z^T K Z (dense Cholesky).
#include <algorithm>
#include <array>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <functional>
#include <mutex>
#include <thread>

#include "factor.h"
#include "geneo.h"

namespace gl {

void fail(int code, const std::string &msg) { throw Error{code, msg}; }

bool is_device_ptr(const void *p) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

static thread_local std::string g_last_error;

// Inverse of a symmetric positive definite 6x6 matrix (Gauss-Jordan).
static void inv6(const double A[36], double X[36]) {
    double a[6][12];
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 12; ++j) a[i][j] = j < 6 ? A[6 * i + j] : (j - 6 == i ? 1.0 : 0.0);
    for (int c = 0; c < 6; ++c) {
        int piv = c;
        for (int r = c + 1; r < 6; ++r)
            if (std::fabs(a[r][c]) > std::fabs(a[piv][c])) piv = r;
        if (std::fabs(a[piv][c]) < 1e-300) fail(GL_ERR_INVALID_ARG, "singular material compliance");
        if (piv != c)
            for (int j = 0; j < 12; ++j) std::swap(a[c][j], a[piv][j]);
        double d = a[c][c];
        for (int j = 0; j < 12; ++j) a[c][j] /= d;
        for (int r = 0; r < 6; ++r)
            if (r != c) {
                double f = a[r][c];
                for (int j = 0; j < 12; ++j) a[r][j] -= f * a[c][j];
            }
    }
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) X[6 * i + j] = a[i][j + 6];
}

static std::vector<std::pair<int, int>> split_range(int n, int p) {
    std::vector<std::pair<int, int>> out;
    int q = n / p, r = n % p, s = 0;
    for (int i = 0; i < p; ++i) {
        int size = q + (i < r ? 1 : 0);
        out.push_back({s, s + size});
        s += size;
    }
    return out;
}

template <class F>
static void parallel_for(int n, F fn) {
    int nt = std::max(1u, std::min(std::thread::hardware_concurrency(), 32u));
    nt = std::min(nt, n);
    std::atomic<int> next(0);
    std::vector<std::thread> th;
    std::vector<Error> errs;
    std::mutex mu;
    bool failed = false;
    for (int t = 0; t < nt; ++t)
        th.emplace_back([&]() {
            for (;;) {
                int i = next++;
                if (i >= n) break;
                try {
                    fn(i);
                } catch (const Error &e) {
                    std::lock_guard<std::mutex> g(mu);
                    errs.push_back(e);
                    failed = true;
                }
            }
        });
    for (auto &t : th) t.join();
    if (failed) throw errs.front();
}

}  // namespace gl

using namespace gl;

namespace {
// Nested dissection stops at regions of at most this many nodes (fewer factor
// entries than larger leaves on the laminate subdomains: 66M against 83M per
// 6x9x92-element subdomain at 125).
constexpr int LEAF_NODES = 64;
std::atomic<long long> g_launches(0);   // kernels launched by gl_solve / gl_apply_* (hot path)
enum { PH_KU = 0, PH_LOCAL = 1, PH_COARSE = 2, PH_N = 3 };
struct Prof {
    bool on = false;
    cudaEvent_t ev[2 * PH_N] = {};
    double ms[PH_N] = {0, 0, 0};
    long long count[PH_N] = {0, 0, 0};
    int pending[PH_N] = {0, 0, 0};
};
}  // namespace

struct gl_ctx {
    Prof prof;
    int device = 0;
    cudaStream_t stream = 0;
    // materials (host, 36 per entry) and kind
    std::vector<double> matC;
    std::vector<uint8_t> mat_iso;
    bool have_mat = false, have_mesh = false, ready = false;
    MeshHost m;
    std::vector<double> psi_x;
    // device mesh data
    DBuf<double> d_tn, d_ln, d_rn, d_X, d_C, d_geo, d_psi, d_theta, d_layer_angle, d_matC;
    DBuf<int> d_layer_of_ez, d_layer_mat;
    DBuf<uint8_t> d_resin;
    // boundary data
    std::vector<int64_t> dir_dof;
    std::vector<double> dir_val;
    DBuf<int64_t> d_dir_dof;
    DBuf<double> d_dir_val;
    std::vector<std::pair<int, std::array<double, 3>>> tractions;
    DBuf<double> d_ftrac;
    // solver
    gl_opts opts{};
    std::vector<SubBox> boxes;
    FactorPlan PD, PN;
    DBuf<double> LD64;
    DBuf<float> LD32;
    DBuf<double> Z;      // coarse basis, Neumann-local layout, m columns
    int m_coarse = 0, n0 = 0;
    DBuf<double> L0;     // K_0 during setup, then K_0^{-1} (dense, from its Cholesky factorisation)
    DBuf<double> cvec2;
    std::vector<double> eig;
    int eig_iters_done = 0;
    // work
    DBuf<double> x, r, z, p, q, ud, fe, partials, cvec, xl64;
    DBuf<float> xl32;
    DBuf<CGScalars> S;
    DBuf<int> err;
    double *h_pin = nullptr;
    double ms_setup = 0;
    int64_t n_free = 0;

    ~gl_ctx() {
        if (h_pin) cudaFreeHost(h_pin);
    }
};

namespace {

int guard(const std::function<void()> &fn) {
    try {
        fn();
        return GL_OK;
    } catch (const Error &e) {
        g_last_error = e.msg;
        return e.code;
    } catch (const std::bad_alloc &) {
        g_last_error = "host out of memory";
        return GL_ERR_OOM;
    } catch (const std::exception &e) {
        g_last_error = e.what();
        return GL_ERR_CUDA;
    }
}

void require_ctx(gl_ctx *c) {
    if (!c) fail(GL_ERR_INVALID_ARG, "null context");
    GL_CUDA(cudaSetDevice(c->device));
}

// Copy n doubles from a caller pointer (host or device) into device memory.
void to_device(double *dst, const double *src, int64_t n, cudaStream_t s) {
    if (n) GL_CUDA(cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyDefault, s));
}
void from_device(double *dst, const double *src, int64_t n, cudaStream_t s) {
    if (n) GL_CUDA(cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyDefault, s));
    GL_CUDA(cudaStreamSynchronize(s));
}

void check_err(gl_ctx *c, const char *what) {
    int h = 0;
    GL_CUDA(cudaMemcpyAsync(&h, c->err.p, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    GL_CUDA(cudaStreamSynchronize(c->stream));
    if (h) {
        c->err.zero(c->stream);
        fail(GL_ERR_NOT_SPD, std::string(what) + ": non-positive pivot");
    }
}

// Setup phase timing to stderr when GL_VERBOSE is set (syncs the stream).
void stamp(gl_ctx *c, const char *what) {
    static const bool on = std::getenv("GL_VERBOSE") != nullptr;
    static thread_local std::chrono::steady_clock::time_point last = std::chrono::steady_clock::now();
    if (!on) return;
    GL_CUDA(cudaStreamSynchronize(c->stream));
    auto now = std::chrono::steady_clock::now();
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    std::fprintf(stderr, "[gl] %-34s %9.3f s   device used %.1f GB\n", what,
                 std::chrono::duration<double>(now - last).count(), (tot - fr) / 1e9);
    last = now;
}

// ---------------------------------------------------------------- geometry + material

void build_geometry(gl_ctx *c) {
    MeshHost &m = c->m;
    cudaStream_t s = c->stream;
    c->d_tn.upload(m.tn, s);
    c->d_ln.upload(m.ln, s);
    c->d_rn.upload(m.rn, s);
    c->d_X.alloc(3 * m.n_nodes);
    launch_node_coords(m, c->d_tn.p, c->d_ln.p, c->d_rn.p, c->d_X.p, s);
    c->psi_x.assign(m.nx, 0.0);
    if (m.geometry == 1)
        for (int ex = 0; ex < m.nx; ++ex) {
            double tc = 0.5 * (m.sv[ex] + m.sv[ex + 1]);
            c->psi_x[ex] = std::min(std::max(tc, 0.0), 1.0) * m.arc_rad;
        }
    c->d_psi.upload(c->psi_x, s);
    c->d_layer_of_ez.upload(m.layer_of_ez, s);
    c->d_layer_mat.upload(m.layer_mat, s);
    c->d_layer_angle.upload(m.layer_angle, s);
    if (!m.theta.empty()) c->d_theta.upload(m.theta, s);
    else c->d_theta.release();
    c->d_matC.upload(c->matC, s);
    c->d_C.alloc(36 * m.n_elem);
    launch_elem_material(m.n_elem, m.nx, m.ny, c->d_layer_of_ez.p, c->d_layer_mat.p, c->d_layer_angle.p,
                         c->d_theta.p, c->d_psi.p, c->d_matC.p, c->d_C.p, s);
    c->d_geo.alloc(270 * m.n_elem);
    launch_elem_geometry(m, c->d_X.p, c->d_geo.p, s);
    std::vector<uint8_t> resin(m.n_elem);
    for (int64_t e = 0; e < m.n_elem; ++e) {
        int ez = (int)(e / ((int64_t)m.nx * m.ny));
        resin[e] = c->mat_iso[m.layer_mat[m.layer_of_ez[ez]]];
    }
    c->d_resin.upload(resin, s);
    c->d_ftrac.alloc(m.n_dof);
    c->d_ftrac.zero(s);
    for (auto &t : c->tractions) launch_traction(m, c->d_X.p, t.first, t.second.data(), c->d_ftrac.p, s);
    GL_CUDA(cudaStreamSynchronize(s));
}

// ---------------------------------------------------------------- decomposition

void build_boxes(gl_ctx *c) {
    const MeshHost &m = c->m;
    const gl_opts &o = c->opts;
    auto rx = split_range(m.nx, o.px), ry = split_range(m.ny, o.py), rz = split_range(m.nz, o.pz);
    const int ne[3] = {m.nx, m.ny, m.nz};
    c->boxes.clear();
    for (int kz = 0; kz < o.pz; ++kz)
        for (int ky = 0; ky < o.py; ++ky)
            for (int kx = 0; kx < o.px; ++kx) {
                SubBox b{};
                std::pair<int, int> core[3] = {rx[kx], ry[ky], rz[kz]};
                for (int d = 0; d < 3; ++d) {
                    int lo = std::max(0, core[d].first - o.overlap), hi = std::min(ne[d], core[d].second + o.overlap);
                    b.ebox[2 * d] = lo;
                    b.ebox[2 * d + 1] = hi;
                    b.nbox[2 * d] = 2 * lo;
                    b.nbox[2 * d + 1] = 2 * hi;
                    b.art[2 * d] = lo > 0;
                    b.art[2 * d + 1] = hi < ne[d];
                }
                c->boxes.push_back(b);
            }
}

// Element -> local index maps of one plan's subdomains.
void build_local_elems(const MeshHost &m, const std::vector<SubBox> &boxes, const FactorPlan &P, LocalElems &E,
                       cudaStream_t s) {
    std::vector<int> elem, sub, loc;
    for (int j = 0; j < P.n_sub; ++j) {
        const SubBox &b = boxes[j];
        const int nbx = b.nbox[1] - b.nbox[0] + 1, nby = b.nbox[3] - b.nbox[2] + 1, nbz = b.nbox[5] - b.nbox[4] + 1;
        std::vector<int> map((size_t)nbx * nby * nbz * 3, -1);
        const int64_t off = P.vec_off[j];
        for (int64_t i = 0; i < P.vec_len[j]; ++i) {
            int64_t g = P.h_gdof[off + i];
            int64_t node = g / 3;
            int comp = (int)(g % 3);
            int x = (int)(node % m.NX), y = (int)((node / m.NX) % m.NY), z = (int)(node / ((int64_t)m.NX * m.NY));
            map[3 * ((size_t)(x - b.nbox[0]) + (size_t)nbx * ((y - b.nbox[2]) + (size_t)nby * (z - b.nbox[4]))) + comp] =
                (int)i;
        }
        for (int ez = b.ebox[4]; ez < b.ebox[5]; ++ez)
            for (int ey = b.ebox[2]; ey < b.ebox[3]; ++ey)
                for (int ex = b.ebox[0]; ex < b.ebox[1]; ++ex) {
                    elem.push_back((int)(ex + (int64_t)m.nx * (ey + (int64_t)m.ny * ez)));
                    sub.push_back(j);
                    for (int a = 0; a < 27; ++a) {
                        int x = 2 * ex + a % 3 - b.nbox[0], y = 2 * ey + (a / 3) % 3 - b.nbox[2],
                            z = 2 * ez + a / 9 - b.nbox[4];
                        for (int cc = 0; cc < 3; ++cc)
                            loc.push_back(map[3 * ((size_t)x + (size_t)nbx * (y + (size_t)nby * z)) + cc]);
                    }
                }
    }
    E.n_pairs = (int64_t)elem.size();
    E.elem.upload(elem, s);
    E.sub.upload(sub, s);
    E.loc.upload(loc, s);
    GL_CUDA(cudaStreamSynchronize(s));
}

// Copies the first m of k columns of a multi-vector (per-subdomain layout).
__global__ void k_copy_cols(const int64_t *__restrict__ voff, const int64_t *__restrict__ vlen,
                            const double *__restrict__ X, int k, double *__restrict__ Y, int mcols) {
    const int s = blockIdx.x;
    const int64_t n = vlen[s];
    for (int64_t i = (int64_t)blockIdx.y * blockDim.x + threadIdx.x; i < n * mcols; i += (int64_t)gridDim.y * blockDim.x) {
        int64_t a = i / n, r = i % n;
        Y[voff[s] * mcols + a * n + r] = X[voff[s] * k + a * n + r];
    }
}

// G (N x m, column stride N) [gdof_j[i], :] (+)= Y_j[i, :]
__global__ void k_scatter_cols(const int64_t *__restrict__ gdof, int64_t off, int64_t n, const double *__restrict__ Y,
                               int64_t yoff, int m, double *__restrict__ G, int64_t N, int zero) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n * m; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t a = i / n, r = i % n;
        G[a * N + gdof[off + r]] = zero ? 0.0 : Y[yoff + a * n + r];
    }
}

// K0[(l*m + a) + (j*m + b) * n0] = sum_i Z_l[i, a] G[gdof_l[i], b]
__global__ void __launch_bounds__(256) k_coarse_block(const int64_t *__restrict__ gdof, int64_t off, int64_t n,
                                                      const double *__restrict__ Z, int64_t zoff, int m,
                                                      const double *__restrict__ G, int64_t N, double *__restrict__ K0,
                                                      int64_t n0, int row0, int col0) {
    const int a = blockIdx.x / m, b = blockIdx.x % m;
    double v = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) v += Z[zoff + a * n + i] * G[b * N + gdof[off + i]];
    __shared__ double red[256];
    red[threadIdx.x] = v;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) K0[(row0 + a) + (int64_t)(col0 + b) * n0] = red[0];
}

void build_geneo(gl_ctx *c, const std::vector<uint8_t> &is_dir) {
    const MeshHost &m = c->m;
    cudaStream_t s = c->stream;
    const int nev = c->opts.nev;
    const double sigma = c->opts.sigma > 0 ? c->opts.sigma : 1e-3;
    const int nsub = (int)c->boxes.size();
    // Neumann symbolic: all free DOFs of each closed subdomain
    std::vector<SubSymbolic> syms(nsub);
    parallel_for(nsub, [&](int j) { build_symbolic(m, c->boxes[j], is_dir, true, LEAF_NODES, syms[j]); });
    build_plan(syms, c->PN, s);
    stamp(c, "Neumann symbolic");
    FactorPlan &PN = c->PN;
    for (int j = 0; j < nsub; ++j)
        if (PN.vec_len[j] < nev) fail(GL_ERR_INVALID_ARG, "subdomain has fewer DOFs than nev");
    // partition of unity: 1/multiplicity over the Dirichlet (interior) sets, 0 on artificial boundaries
    std::vector<int> mult(m.n_dof, 0);
    for (int64_t g : c->PD.h_gdof) mult[g] += 1;
    std::vector<double> xi(PN.n_local, 0.0);
    for (int j = 0; j < nsub; ++j) {
        const SubBox &b = c->boxes[j];
        for (int64_t i = 0; i < PN.vec_len[j]; ++i) {
            int64_t g = PN.h_gdof[PN.vec_off[j] + i];
            int64_t node = g / 3;
            int pos[3] = {(int)(node % m.NX), (int)((node / m.NX) % m.NY), (int)(node / ((int64_t)m.NX * m.NY))};
            bool art = false;
            for (int d = 0; d < 3; ++d) {
                if (b.art[2 * d] && pos[d] == b.nbox[2 * d]) art = true;
                if (b.art[2 * d + 1] && pos[d] == b.nbox[2 * d + 1]) art = true;
            }
            if (!art) {
                if (mult[g] == 0) fail(GL_ERR_INVALID_ARG, "a free DOF lies in no subdomain interior (overlap >= 1?)");
                xi[PN.vec_off[j] + i] = 1.0 / mult[g];
            }
        }
    }
    DBuf<double> d_xi;
    d_xi.upload(xi, s);
    const int k = std::min(32, std::max(nev + 4, ((2 * nev + 3) / 4) * 4));
    const int64_t nl = PN.n_local;
    c->m_coarse = nev;
    c->n0 = nsub * nev;
    c->Z.alloc(nl * nev);
    c->eig.assign((size_t)nsub * nev, 0.0);
    const int iters = c->opts.eig_iters > 0 ? c->opts.eig_iters : 100;
    // Groups of subdomains: factor of A^N + sigma Xi A^N Xi and block subspace
    // iteration for the largest mu of B p = mu M p, one group at a time.
    const int64_t budget = (int64_t)(40e9 / sizeof(double));   // factor entries per group
    int j0 = 0, max_its = 0;
    while (j0 < nsub) {
        int j1 = j0;
        int64_t acc = 0;
        while (j1 < nsub && (j1 == j0 || acc + syms[j1].l_size <= budget)) acc += syms[j1++].l_size;
        const int ng = j1 - j0;
        std::vector<SubSymbolic> gs(syms.begin() + j0, syms.begin() + j1);
        FactorPlan PG;
        build_plan(gs, PG, s);
        gs.clear();
        const int64_t goff = PN.vec_off[j0], gl = PG.n_local;
        DBuf<double> LN;
        LN.alloc(PG.l_size);
        const double *xg = d_xi.p + goff;
        numeric_factor<double>(PG, c->d_C.p, c->d_geo.p, xg, sigma, LN.p, c->err.p, s);
        check_err(c, "GenEO shifted Neumann factorisation");
        stamp(c, "Neumann factorisation (group)");
        std::vector<SubBox> gboxes(c->boxes.begin() + j0, c->boxes.begin() + j1);
        LocalElems E;
        build_local_elems(m, gboxes, PG, E, s);
        DBuf<double> V, BV, BW, tmp, GB, GM, Y, mu;
        V.alloc(gl * k);
        BV.alloc(gl * k);
        BW.alloc(gl * k);
        tmp.alloc(gl * k);
        GB.alloc((size_t)ng * k * k);
        GM.alloc((size_t)ng * k * k);
        Y.alloc((size_t)ng * k * k);
        mu.alloc((size_t)ng * k);
        fill_random(V.p, gl * k, 0x1707042280000001ull + (uint64_t)j0, s);
        BV.zero(s);
        local_K_apply(PG, E, c->d_C.p, c->d_geo.p, xg, V.p, BV.p, k, s);          // BV = Xi A^N Xi V
        std::vector<double> mu_prev((size_t)ng * k, 0.0), mu_now((size_t)ng * k);
        int it = 0;
        for (; it < iters; ++it) {
            // W = M^{-1} B V
            GL_CUDA(cudaMemcpyAsync(tmp.p, BV.p, sizeof(double) * gl * k, cudaMemcpyDeviceToDevice, s));
            factor_solve<double>(PG, LN.p, tmp.p, k, s);
            std::swap(V.p, tmp.p);
            BW.zero(s);
            local_K_apply(PG, E, c->d_C.p, c->d_geo.p, xg, V.p, BW.p, k, s);       // BW = B W
            local_gram(PG, V.p, BV.p, k, GM.p, s);                  // W^T M W = W^T (B V)
            local_gram(PG, V.p, BW.p, k, GB.p, s);                  // W^T B W
            small_geneig(ng, k, GB.p, GM.p, Y.p, mu.p, c->err.p, s);
            check_err(c, "GenEO Rayleigh-Ritz");
            local_rotate(PG, V.p, Y.p, k, tmp.p, s);
            local_rotate(PG, BW.p, Y.p, k, tmp.p, s);
            std::swap(BV.p, BW.p);
            GL_CUDA(cudaMemcpyAsync(mu_now.data(), mu.p, mu_now.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
            GL_CUDA(cudaStreamSynchronize(s));
            double change = 0.0;
            for (int j = 0; j < ng; ++j)
                for (int a = 0; a < nev; ++a) {
                    double now = mu_now[(size_t)j * k + a], prev = mu_prev[(size_t)j * k + a];
                    change = std::max(change, std::fabs(now - prev) / std::fabs(now));
                }
            mu_prev = mu_now;
            // Ritz values settle to ~(rate)^{2 it}; 1e-12 leaves the Ritz vectors accurate to
            // about 1e-6, far below what changes the coarse space's effect on PCG.
            if (it >= 4 && change < 1e-12) {
                ++it;
                break;
            }
        }
        if (std::getenv("GL_VERBOSE")) {
            double worst = 0.0, lo = 1e300, hi = 0.0;
            for (int j = 0; j < ng; ++j) {
                double lm = 1.0 / mu_now[(size_t)j * k + nev - 1] - sigma, lk = 1.0 / mu_now[(size_t)j * k + k - 1] - sigma;
                worst = std::max(worst, (lm + sigma) / (lk + sigma));
                lo = std::min(lo, lm);
                hi = std::max(hi, lm);
            }
            std::fprintf(stderr, "[gl]   group %d-%d: %d iterations, lambda_nev in [%.3g, %.3g], worst rate %.3f\n", j0,
                         j1 - 1, it, lo, hi, worst);
        }
        max_its = std::max(max_its, it);
        for (int j = 0; j < ng; ++j)
            for (int a = 0; a < nev; ++a) c->eig[(size_t)(j0 + j) * nev + a] = 1.0 / mu_now[(size_t)j * k + a] - sigma;
        // Z columns of these subdomains (global Neumann layout, nev columns)
        for (int j = 0; j < ng; ++j) {
            const int64_t n = PG.vec_len[j];
            GL_CUDA(cudaMemcpy2DAsync(c->Z.p + PN.vec_off[j0 + j] * nev, n * sizeof(double), V.p + PG.vec_off[j] * k,
                                      n * sizeof(double), n * sizeof(double), nev, cudaMemcpyDeviceToDevice, s));
        }
        stamp(c, "GenEO subspace iteration (group)");
        j0 = j1;
    }
    c->eig_iters_done = max_its;
    if (std::getenv("GL_VERBOSE")) std::fprintf(stderr, "[gl] GenEO subspace iterations (max over groups): %d\n", max_its);
    syms.clear();
    scale_rows(PN, c->Z.p, d_xi.p, nev, s);                        // Z = Xi p
    LocalElems E;
    build_local_elems(m, c->boxes, PN, E, s);
    // K_0 = Z^T K Z: Y_j = A^N_j Z_j, then blocks against overlapping subdomains
    DBuf<double> KZ, G;
    KZ.alloc(nl * nev);
    KZ.zero(s);
    local_K_apply(PN, E, c->d_C.p, c->d_geo.p, nullptr, c->Z.p, KZ.p, nev, s);
    G.alloc((size_t)m.n_dof * nev);
    G.zero(s);
    const int n0 = c->n0;
    c->L0.alloc((size_t)n0 * n0);
    c->L0.zero(s);
    for (int j = 0; j < nsub; ++j) {
        int64_t nj = PN.vec_len[j], oj = PN.vec_off[j];
        k_scatter_cols<<<256, 256, 0, s>>>(PN.d_gdof.p, oj, nj, KZ.p, oj * nev, nev, G.p, m.n_dof, 0);
        for (int l = 0; l < nsub; ++l) {
            bool overlap = true;
            for (int d = 0; d < 3; ++d)
                if (c->boxes[l].nbox[2 * d] > c->boxes[j].nbox[2 * d + 1] ||
                    c->boxes[j].nbox[2 * d] > c->boxes[l].nbox[2 * d + 1])
                    overlap = false;
            if (!overlap) continue;
            k_coarse_block<<<nev * nev, 256, 0, s>>>(PN.d_gdof.p, PN.vec_off[l], PN.vec_len[l], c->Z.p,
                                                     PN.vec_off[l] * nev, nev, G.p, m.n_dof, c->L0.p, n0, l * nev,
                                                     j * nev);
        }
        k_scatter_cols<<<256, 256, 0, s>>>(PN.d_gdof.p, oj, nj, KZ.p, oj * nev, nev, G.p, m.n_dof, 1);
        GL_CUDA(cudaGetLastError());
    }
    {
        DBuf<double> K0inv;
        K0inv.alloc((size_t)n0 * n0);
        dense_inverse(c->L0.p, n0, K0inv.p, c->err.p, s);
        c->L0 = std::move(K0inv);
    }
    check_err(c, "coarse Cholesky");
    GL_CUDA(cudaStreamSynchronize(s));
}

// ---------------------------------------------------------------- operator pieces

// Per-phase CUDA-event timing (only when profiling is on).  Each phase keeps
// one start/stop pair; a pending pair is folded into the totals before reuse.
void prof_fold(gl_ctx *c, int ph) {
    Prof &P = c->prof;
    if (!P.pending[ph]) return;
    GL_CUDA(cudaEventSynchronize(P.ev[2 * ph + 1]));
    float ms = 0;
    GL_CUDA(cudaEventElapsedTime(&ms, P.ev[2 * ph], P.ev[2 * ph + 1]));
    P.ms[ph] += ms;
    P.count[ph] += 1;
    P.pending[ph] = 0;
}
void prof_begin(gl_ctx *c, int ph) {
    if (!c->prof.on) return;
    prof_fold(c, ph);
    GL_CUDA(cudaEventRecord(c->prof.ev[2 * ph], c->stream));
}
void prof_end(gl_ctx *c, int ph) {
    if (!c->prof.on) return;
    GL_CUDA(cudaEventRecord(c->prof.ev[2 * ph + 1], c->stream));
    c->prof.pending[ph] = 1;
}

int64_t factor_solve_launches(const FactorPlan &P) {
    int64_t n = 0;
    for (auto &L : P.levels)
        if (!L.fronts.empty()) n += 2;
    return n;
}

void apply_K(gl_ctx *c, const double *x, double *y) {
    prof_begin(c, PH_KU);
    launch_ku(c->m, c->d_C.p, c->d_geo.p, x, y, c->stream);
    prof_end(c, PH_KU);
    g_launches += 1;
}

// z = M^{-1} r (r zero at Dirichlet DOFs)
void apply_prec(gl_ctx *c, const double *r, double *z) {
    cudaStream_t s = c->stream;
    GL_CUDA(cudaMemsetAsync(z, 0, c->m.n_dof * sizeof(double), s));
    prof_begin(c, PH_LOCAL);
    if (c->opts.precision == GL_PREC_MIXED) {
        gather_local<float>(c->PD, r, c->xl32.p, s);
        factor_solve<float>(c->PD, c->LD32.p, c->xl32.p, 1, s);
        scatter_add_local<float>(c->PD, c->xl32.p, z, s);
    } else {
        gather_local<double>(c->PD, r, c->xl64.p, s);
        factor_solve<double>(c->PD, c->LD64.p, c->xl64.p, 1, s);
        scatter_add_local<double>(c->PD, c->xl64.p, z, s);
    }
    prof_end(c, PH_LOCAL);
    g_launches += 2 + factor_solve_launches(c->PD);
    if (c->n0 > 0) {
        prof_begin(c, PH_COARSE);
        coarse_restrict(c->PN, c->Z.p, c->m_coarse, r, c->cvec.p, s);
        dense_symv(c->L0.p, c->n0, c->cvec.p, c->cvec2.p, s);
        coarse_prolong(c->PN, c->Z.p, c->m_coarse, c->cvec2.p, z, s);
        prof_end(c, PH_COARSE);
        g_launches += 3;
    }
}

void setup(gl_ctx *c, const gl_opts &o) {
    auto t0 = std::chrono::steady_clock::now();
    if (!c->have_mat || !c->have_mesh) fail(GL_ERR_STATE, "gl_setup: materials and mesh must be set first");
    GL_REQUIRE(o.px >= 1 && o.py >= 1 && o.pz >= 1, "subdomain counts must be >= 1");
    GL_REQUIRE(o.overlap >= 1, "overlap must be >= 1");
    GL_REQUIRE(o.nev >= 0 && o.nev <= 28, "nev must be in [0, 28]");
    GL_REQUIRE(o.px <= c->m.nx && o.py <= c->m.ny && o.pz <= c->m.nz, "more subdomains than elements along an axis");
    GL_REQUIRE(o.precision == GL_PREC_FP64 || o.precision == GL_PREC_MIXED, "unknown precision mode");
    c->ready = false;
    c->opts = o;
    if (c->opts.max_iter <= 0) c->opts.max_iter = 2000;
    if (c->opts.tol <= 0) c->opts.tol = 1e-10;
    if (c->opts.resid_period <= 0) c->opts.resid_period = 50;
    cudaStream_t s = c->stream;
    const MeshHost &m = c->m;
    if (!c->err.p) {
        c->err.alloc(1);
        c->err.zero(s);
    }
    stamp(c, "start");
    build_geometry(c);
    stamp(c, "geometry, materials, loads");
    std::vector<uint8_t> is_dir(m.n_dof, 0);
    for (int64_t d : c->dir_dof) is_dir[d] = 1;
    c->n_free = m.n_dof - (int64_t)std::count(is_dir.begin(), is_dir.end(), (uint8_t)1);
    build_boxes(c);
    const int nsub = (int)c->boxes.size();
    std::vector<SubSymbolic> syms(nsub);
    parallel_for(nsub, [&](int j) { build_symbolic(m, c->boxes[j], is_dir, false, LEAF_NODES, syms[j]); });
    build_plan(syms, c->PD, s);
    syms.clear();
    stamp(c, "Dirichlet symbolic");
    if (c->opts.precision == GL_PREC_MIXED) {
        c->LD64.release();
        c->LD32.alloc(c->PD.l_size);
        numeric_factor<float>(c->PD, c->d_C.p, c->d_geo.p, nullptr, 0.0, c->LD32.p, c->err.p, s);
    } else {
        c->LD32.release();
        c->LD64.alloc(c->PD.l_size);
        numeric_factor<double>(c->PD, c->d_C.p, c->d_geo.p, nullptr, 0.0, c->LD64.p, c->err.p, s);
    }
    check_err(c, "local Dirichlet factorisation");
    stamp(c, "Dirichlet factorisation");
    c->n0 = 0;
    c->m_coarse = 0;
    c->eig.clear();
    if (c->opts.nev > 0) build_geneo(c, is_dir);
    stamp(c, "GenEO coarse space + K0");
    // work vectors
    const int64_t N = m.n_dof;
    for (DBuf<double> *b : {&c->x, &c->r, &c->z, &c->p, &c->q, &c->ud, &c->fe}) b->alloc(N);
    c->partials.alloc(1024);
    c->cvec.alloc(std::max(1, c->n0));
    c->cvec2.alloc(std::max(1, c->n0));
    if (c->opts.precision == GL_PREC_MIXED) {
        c->xl32.alloc(c->PD.n_local);
        c->xl64.release();
    } else {
        c->xl64.alloc(c->PD.n_local);
        c->xl32.release();
    }
    c->S.alloc(1);
    if (!c->h_pin) GL_CUDA(cudaMallocHost(&c->h_pin, 8 * sizeof(double)));
    GL_CUDA(cudaStreamSynchronize(s));
    c->ready = true;
    c->ms_setup = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

double read_scalar(gl_ctx *c, const double *d) {
    GL_CUDA(cudaMemcpyAsync(c->h_pin, d, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    GL_CUDA(cudaStreamSynchronize(c->stream));
    return c->h_pin[0];
}

// Effective right-hand side fe = f - K u_D on the free DOFs, 0 on Dirichlet DOFs.
void prepare_rhs(gl_ctx *c, const double *f, bool homogeneous) {
    cudaStream_t s = c->stream;
    const int64_t N = c->m.n_dof, nd = (int64_t)c->dir_dof.size();
    if (f) to_device(c->fe.p, f, N, s);
    else GL_CUDA(cudaMemcpyAsync(c->fe.p, c->d_ftrac.p, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
    c->ud.zero(s);
    if (!homogeneous) set_entries(c->ud.p, c->d_dir_dof.p, nd, c->d_dir_val.p, s);
    apply_K(c, c->ud.p, c->q.p);
    sub(c->fe.p, c->fe.p, c->q.p, N, s);
    set_entries(c->fe.p, c->d_dir_dof.p, nd, nullptr, s);
    g_launches += 1 + (nd ? 2 : 0);
}

// PCG solve of K u = f; homogeneous = zero Dirichlet values (adjoint solves).
void solve(gl_ctx *c, const double *f, double *u, gl_info *info, bool homogeneous = false) {
    if (!c->ready) fail(GL_ERR_STATE, "gl_solve before gl_setup");
    cudaStream_t s = c->stream;
    const int64_t N = c->m.n_dof, nd = (int64_t)c->dir_dof.size();
    cudaEvent_t e0, e1;
    GL_CUDA(cudaEventCreate(&e0));
    GL_CUDA(cudaEventCreate(&e1));
    GL_CUDA(cudaEventRecord(e0, s));
    prepare_rhs(c, f, homogeneous);
    CGScalars *S = c->S.p;
    c->S.zero(s);
    dot(c->fe.p, c->fe.p, N, c->partials.p, &S->ff, s);
    const int nds = nd ? 1 : 0;   // set_entries launches a kernel only for a non-empty list
    g_launches += 2;
    const double ff = read_scalar(c, &S->ff);
    if (!std::isfinite(ff)) {
        GL_CUDA(cudaEventDestroy(e0));
        GL_CUDA(cudaEventDestroy(e1));
        fail(GL_ERR_NAN, "non-finite load vector");
    }
    const bool mixed = c->opts.precision == GL_PREC_MIXED;
    c->x.zero(s);
    GL_CUDA(cudaMemcpyAsync(c->r.p, c->fe.p, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
    int iters = 0, status = GL_OK;
    double rel = 0.0;
    if (ff > 0.0) {
        apply_prec(c, c->r.p, c->z.p);
        dot(c->r.p, c->z.p, N, c->partials.p, &S->rho, s);
        g_launches += 2;
        GL_CUDA(cudaMemcpyAsync(c->p.p, c->z.p, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
        rel = 1.0;
        for (int it = 1; it <= c->opts.max_iter; ++it) {
            apply_K(c, c->p.p, c->q.p);
            set_entries(c->q.p, c->d_dir_dof.p, nd, nullptr, s);
            dot(c->p.p, c->q.p, N, c->partials.p, &S->pq, s);
            cg_update_xr(c->x.p, c->r.p, c->p.p, c->q.p, N, S, c->partials.p, s);
            g_launches += nds + 4;
            const double rr = read_scalar(c, &S->rr);
            iters = it;
            if (!std::isfinite(rr)) {
                status = GL_ERR_NAN;
                break;
            }
            rel = std::sqrt(rr / ff);
            // stop on the recurrence residual; the FP64 true residual is reported after the loop
            // (on these laminates its rounding floor lies near 1e-10 * ||K|| ||x|| / ||f||)
            if (rel <= c->opts.tol) break;
            if (it == c->opts.max_iter) {
                status = GL_ERR_NOT_CONVERGED;
                break;
            }
            if (mixed && it % c->opts.resid_period == 0) {
                // residual replacement: r = fe - K x in FP64
                apply_K(c, c->x.p, c->q.p);
                set_entries(c->q.p, c->d_dir_dof.p, nd, nullptr, s);
                sub(c->r.p, c->fe.p, c->q.p, N, s);
                g_launches += nds + 1;
            }
            if (mixed) {
                dot(c->r.p, c->z.p, N, c->partials.p, &S->rz_old, s);   // flexible beta
                g_launches += 2;
            }
            apply_prec(c, c->r.p, c->z.p);
            dot(c->r.p, c->z.p, N, c->partials.p, &S->rho_new, s);
            cg_update_p(c->p.p, c->z.p, N, S, s);
            g_launches += 4;
        }
    }
    // true residual and the full displacement
    apply_K(c, c->x.p, c->q.p);
    set_entries(c->q.p, c->d_dir_dof.p, nd, nullptr, s);
    sub(c->r.p, c->fe.p, c->q.p, N, s);
    dot(c->r.p, c->r.p, N, c->partials.p, &S->rr, s);
    const double rt = read_scalar(c, &S->rr);
    axpy(c->x.p, 1.0, c->ud.p, N, s);
    g_launches += nds + 4;
    for (int ph = 0; ph < PH_N; ++ph) prof_fold(c, ph);
    GL_CUDA(cudaEventRecord(e1, s));
    from_device(u, c->x.p, N, s);
    float ms = 0;
    GL_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (info) {
        info->iters = iters;
        info->status = status;
        info->rel_resid = rel;
        info->rel_resid_true = ff > 0 ? std::sqrt(rt / ff) : 0.0;
        info->ms_setup = c->ms_setup;
        info->ms_solve = ms;
        info->n_free = c->n_free;
        info->n_coarse = c->n0;
        info->factor_nnz = c->PD.l_size;
    }
    if (status != GL_OK) {
        g_last_error = status == GL_ERR_NAN ? "NaN/Inf in the PCG iteration" : "PCG reached max_iter";
        throw Error{status, g_last_error};
    }
}

}  // namespace

// ====================================================================== C ABI

extern "C" {

const char *gl_strerror(int code) {
    switch (code) {
        case GL_OK: return "ok";
        case GL_ERR_INVALID_ARG: return "invalid argument";
        case GL_ERR_OOM: return "out of memory";
        case GL_ERR_CUDA: return "CUDA error";
        case GL_ERR_NOT_SPD: return "matrix not positive definite";
        case GL_ERR_NOT_CONVERGED: return "not converged";
        case GL_ERR_NAN: return "NaN or Inf";
        case GL_ERR_TIMEOUT: return "device wait timed out";
        case GL_ERR_STATE: return "call out of order";
        default: return "unknown error";
    }
}

const char *gl_last_error(void) { return g_last_error.c_str(); }

int gl_create(gl_ctx **out, int device, void *cuda_stream) {
    return guard([&] {
        GL_REQUIRE(out, "null output pointer");
        int n = 0;
        GL_CUDA(cudaGetDeviceCount(&n));
        GL_REQUIRE(device >= 0 && device < n, "no such CUDA device");
        GL_CUDA(cudaSetDevice(device));
        gl_ctx *c = new gl_ctx();
        c->device = device;
        c->stream = (cudaStream_t)cuda_stream;
        *out = c;
    });
}

void gl_destroy(gl_ctx *ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    delete ctx;
}

int gl_set_materials(gl_ctx *c, int n_ortho, const gl_ortho *ortho, int n_iso, const double *E_nu) {
    return guard([&] {
        require_ctx(c);
        GL_REQUIRE(n_ortho >= 0 && n_iso >= 0 && n_ortho + n_iso > 0, "empty material table");
        auto ho = fetch(ortho, n_ortho);
        auto hi = fetch(E_nu, 2 * (size_t)n_iso);
        c->matC.clear();
        c->mat_iso.clear();
        for (auto &o : ho) {
            GL_REQUIRE(o.E1 > 0 && o.E2 > 0 && o.E3 > 0 && o.G12 > 0 && o.G13 > 0 && o.G23 > 0,
                       "orthotropic moduli must be positive");
            double S[36] = {0};
            S[0] = 1 / o.E1; S[7] = 1 / o.E2; S[14] = 1 / o.E3;
            S[1] = S[6] = -o.nu12 / o.E1;
            S[2] = S[12] = -o.nu13 / o.E1;
            S[8] = S[13] = -o.nu23 / o.E2;
            S[21] = 1 / o.G23; S[28] = 1 / o.G13; S[35] = 1 / o.G12;
            double C[36];
            inv6(S, C);
            c->matC.insert(c->matC.end(), C, C + 36);
            c->mat_iso.push_back(0);
        }
        for (int i = 0; i < n_iso; ++i) {
            double E = hi[2 * i], nu = hi[2 * i + 1];
            GL_REQUIRE(E > 0 && nu > -1 && nu < 0.5, "isotropic constants out of range");
            double lam = E * nu / ((1 + nu) * (1 - 2 * nu)), mu = E / (2 * (1 + nu));
            double C[36] = {0};
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) C[6 * a + b] = lam + (a == b ? 2 * mu : 0);
            C[21] = C[28] = C[35] = mu;
            c->matC.insert(c->matC.end(), C, C + 36);
            c->mat_iso.push_back(1);
        }
        c->have_mat = true;
        c->ready = false;
    });
}

int gl_set_mesh(gl_ctx *c, const gl_mesh *mesh) {
    return guard([&] {
        require_ctx(c);
        GL_REQUIRE(mesh, "null mesh");
        GL_REQUIRE(c->have_mat, "gl_set_materials must come before gl_set_mesh");
        GL_REQUIRE(mesh->nx >= 1 && mesh->ny >= 1 && mesh->nlayers >= 1, "empty mesh");
        GL_REQUIRE(mesh->geometry == 0 || mesh->geometry == 1, "geometry must be 0 or 1");
        MeshHost m;
        m.nx = mesh->nx;
        m.ny = mesh->ny;
        m.sv = fetch(mesh->x, m.nx + 1);
        m.lv = fetch(mesh->y, m.ny + 1);
        auto nel = fetch(mesh->layer_nel, mesh->nlayers);
        auto th = fetch(mesh->layer_thick, mesh->nlayers);
        m.layer_mat = fetch(mesh->layer_mat, mesh->nlayers);
        auto ang = fetch(mesh->layer_angle_deg, mesh->nlayers);
        for (int i = 0; i < m.nx; ++i) GL_REQUIRE(m.sv[i + 1] > m.sv[i], "x vertices must increase");
        for (int i = 0; i < m.ny; ++i) GL_REQUIRE(m.lv[i + 1] > m.lv[i], "y vertices must increase");
        m.rv.assign(1, 0.0);
        double base = 0.0;
        for (int k = 0; k < mesh->nlayers; ++k) {
            GL_REQUIRE(nel[k] >= 1 && th[k] > 0, "layers need >= 1 element and positive thickness");
            GL_REQUIRE(m.layer_mat[k] >= 0 && m.layer_mat[k] < (int)c->mat_iso.size(), "layer material out of range");
            for (int i = 0; i < nel[k]; ++i) {
                m.rv.push_back(base + th[k] * (i + 1) / nel[k]);
                m.layer_of_ez.push_back(k);
            }
            base += th[k];
            m.layer_angle.push_back(ang[k] * M_PI / 180.0);
        }
        m.nz = (int)m.layer_of_ez.size();
        m.NX = 2 * m.nx + 1;
        m.NY = 2 * m.ny + 1;
        m.NZ = 2 * m.nz + 1;
        m.n_nodes = (int64_t)m.NX * m.NY * m.NZ;
        m.n_dof = 3 * m.n_nodes;
        m.n_elem = (int64_t)m.nx * m.ny * m.nz;
        GL_REQUIRE(m.n_dof < (int64_t)1 << 31, "mesh too large for 32-bit local indices");
        m.geometry = mesh->geometry;
        m.R_inner = mesh->R_inner;
        m.limb_L = mesh->limb_L;
        m.arc_rad = mesh->arc_deg * M_PI / 180.0;
        if (m.geometry == 1) GL_REQUIRE(m.R_inner > 0 && m.arc_rad > 0, "curved mesh needs R_inner > 0, arc > 0");
        auto mid = [](const std::vector<double> &v) {
            std::vector<double> o(2 * v.size() - 1);
            for (size_t i = 0; i < v.size(); ++i) o[2 * i] = v[i];
            for (size_t i = 0; i + 1 < v.size(); ++i) o[2 * i + 1] = 0.5 * (v[i] + v[i + 1]);
            return o;
        };
        m.tn = mid(m.sv);
        m.ln = mid(m.lv);
        m.rn = mid(m.rv);
        if (mesh->theta_e) m.theta = fetch(mesh->theta_e, m.n_elem);
        c->m = std::move(m);
        c->have_mesh = true;
        c->ready = false;
        c->dir_dof.clear();
        c->dir_val.clear();
        c->tractions.clear();
    });
}

int gl_set_dirichlet(gl_ctx *c, int64_t n, const int64_t *dof, const double *val) {
    return guard([&] {
        require_ctx(c);
        GL_REQUIRE(c->have_mesh, "gl_set_mesh must come first");
        GL_REQUIRE(n >= 0, "negative count");
        auto d = fetch(dof, n);
        auto v = fetch(val, n);
        std::vector<std::pair<int64_t, double>> pv;
        for (int64_t i = 0; i < n; ++i) {
            GL_REQUIRE(d[i] >= 0 && d[i] < c->m.n_dof, "Dirichlet DOF out of range");
            pv.push_back({d[i], v[i]});
        }
        std::sort(pv.begin(), pv.end());
        c->dir_dof.clear();
        c->dir_val.clear();
        for (auto &q : pv) {
            if (!c->dir_dof.empty() && c->dir_dof.back() == q.first) {
                c->dir_val.back() = q.second;
                continue;
            }
            c->dir_dof.push_back(q.first);
            c->dir_val.push_back(q.second);
        }
        c->d_dir_dof.upload(c->dir_dof, c->stream);
        c->d_dir_val.upload(c->dir_val, c->stream);
        GL_CUDA(cudaStreamSynchronize(c->stream));
        c->ready = false;
    });
}

int gl_set_traction(gl_ctx *c, int face, const double t[3]) {
    return guard([&] {
        require_ctx(c);
        GL_REQUIRE(c->have_mesh, "gl_set_mesh must come first");
        GL_REQUIRE(face >= 0 && face < 6, "face must be in 0..5");
        auto h = fetch(t, 3);
        c->tractions.push_back({face, {h[0], h[1], h[2]}});
        c->ready = false;
    });
}

int gl_setup(gl_ctx *c, const gl_opts *o) {
    return guard([&] {
        require_ctx(c);
        GL_REQUIRE(o, "null options");
        setup(c, *o);
    });
}

int gl_num_dofs(const gl_ctx *c, int64_t *n) {
    return guard([&] {
        GL_REQUIRE(c && n && c->have_mesh, "no mesh");
        *n = c->m.n_dof;
    });
}

int gl_num_elems(const gl_ctx *c, int64_t *n) {
    return guard([&] {
        GL_REQUIRE(c && n && c->have_mesh, "no mesh");
        *n = c->m.n_elem;
    });
}

int gl_rhs(gl_ctx *c, double *f) {
    return guard([&] {
        require_ctx(c);
        if (!c->ready) fail(GL_ERR_STATE, "gl_rhs before gl_setup");
        GL_REQUIRE(f, "null output");
        from_device(f, c->d_ftrac.p, c->m.n_dof, c->stream);
    });
}

int gl_solve(gl_ctx *c, const double *f, double *u, gl_info *info) {
    return guard([&] {
        require_ctx(c);
        GL_REQUIRE(u, "null output");
        solve(c, f, u, info);
    });
}

int gl_stress(gl_ctx *c, const double *u, double *s33, double *t13, double *peak) {
    return guard([&] {
        require_ctx(c);
        if (!c->ready) fail(GL_ERR_STATE, "gl_stress before gl_setup");
        GL_REQUIRE(u, "null displacement");
        cudaStream_t s = c->stream;
        const MeshHost &m = c->m;
        DBuf<double> du, d33, d13, dpk;
        du.alloc(m.n_dof);
        to_device(du.p, u, m.n_dof, s);
        d33.alloc(m.n_elem);
        d13.alloc(m.n_elem);
        launch_stress(m, c->d_X.p, c->d_C.p, c->d_psi.p, du.p, d33.p, d13.p, s);
        g_launches += 1 + (peak ? 1 : 0);
        if (s33) from_device(s33, d33.p, m.n_elem, s);
        if (t13) from_device(t13, d13.p, m.n_elem, s);
        if (peak) {
            dpk.alloc(1);
            max_where(d33.p, c->d_resin.p, m.n_elem, dpk.p, s);
            from_device(peak, dpk.p, 1, s);
        }
        GL_CUDA(cudaStreamSynchronize(s));
    });
}

int gl_apply_K(gl_ctx *c, const double *x, double *y) {
    return guard([&] {
        require_ctx(c);
        if (!c->ready) fail(GL_ERR_STATE, "gl_apply_K before gl_setup");
        GL_REQUIRE(x && y, "null vector");
        cudaStream_t s = c->stream;
        to_device(c->p.p, x, c->m.n_dof, s);
        apply_K(c, c->p.p, c->q.p);
        from_device(y, c->q.p, c->m.n_dof, s);
    });
}

int gl_apply_prec(gl_ctx *c, const double *r, double *z) {
    return guard([&] {
        require_ctx(c);
        if (!c->ready) fail(GL_ERR_STATE, "gl_apply_prec before gl_setup");
        GL_REQUIRE(r && z, "null vector");
        cudaStream_t s = c->stream;
        to_device(c->r.p, r, c->m.n_dof, s);
        set_entries(c->r.p, c->d_dir_dof.p, (int64_t)c->dir_dof.size(), nullptr, s);
        apply_prec(c, c->r.p, c->z.p);
        from_device(z, c->z.p, c->m.n_dof, s);
    });
}

int gl_set_theta(gl_ctx *c, const double *theta_e) {
    return guard([&] {
        require_ctx(c);
        GL_REQUIRE(c->have_mesh, "gl_set_mesh must come first");
        GL_REQUIRE(theta_e, "null theta");
        MeshHost &m = c->m;
        m.theta = fetch(theta_e, m.n_elem);
        if (c->ready) {
            // new C_e for K u and the stresses; the factors and the coarse space are kept
            c->d_theta.upload(m.theta, c->stream);
            launch_elem_material(m.n_elem, m.nx, m.ny, c->d_layer_of_ez.p, c->d_layer_mat.p, c->d_layer_angle.p,
                                 c->d_theta.p, c->d_psi.p, c->d_matC.p, c->d_C.p, c->stream);
            GL_CUDA(cudaStreamSynchronize(c->stream));
        }
    });
}

int gl_stress_vjp(gl_ctx *c, const double *u, const double *w33, const double *w13, double *dJdu, double *dJdth) {
    return guard([&] {
        require_ctx(c);
        if (!c->ready) fail(GL_ERR_STATE, "gl_stress_vjp before gl_setup");
        GL_REQUIRE(u, "null displacement");
        cudaStream_t s = c->stream;
        const MeshHost &m = c->m;
        DBuf<double> du, d33, d13, dgu, dgt;
        du.alloc(m.n_dof);
        to_device(du.p, u, m.n_dof, s);
        if (w33) {
            d33.alloc(m.n_elem);
            to_device(d33.p, w33, m.n_elem, s);
        }
        if (w13) {
            d13.alloc(m.n_elem);
            to_device(d13.p, w13, m.n_elem, s);
        }
        if (dJdu) {
            dgu.alloc(m.n_dof);
            dgu.zero(s);
        }
        if (dJdth) dgt.alloc(m.n_elem);
        launch_stress_vjp(m, c->d_X.p, c->d_C.p, c->d_psi.p, c->d_layer_of_ez.p, c->d_layer_mat.p,
                          c->d_layer_angle.p, c->d_theta.p, c->d_matC.p, du.p, d33.p, d13.p, dgu.p, dgt.p, s);
        g_launches += 1;
        if (dJdu) from_device(dJdu, dgu.p, m.n_dof, s);
        if (dJdth) from_device(dJdth, dgt.p, m.n_elem, s);
        GL_CUDA(cudaStreamSynchronize(s));
    });
}

int gl_adjoint(gl_ctx *c, const double *u, const double *dJdu, double *grad, gl_info *info) {
    return guard([&] {
        require_ctx(c);
        if (!c->ready) fail(GL_ERR_STATE, "gl_adjoint before gl_setup");
        GL_REQUIRE(u && dJdu && grad, "null argument");
        cudaStream_t s = c->stream;
        const MeshHost &m = c->m;
        DBuf<double> lam, du, dg;
        lam.alloc(m.n_dof);
        solve(c, dJdu, lam.p, info, true);          // K_ff lambda = (dJ/du)_f, lambda = 0 on Dirichlet DOFs
        du.alloc(m.n_dof);
        to_device(du.p, u, m.n_dof, s);
        dg.alloc(m.n_elem);
        launch_adjoint_contract(m, c->d_geo.p, c->d_layer_of_ez.p, c->d_layer_mat.p, c->d_layer_angle.p,
                                c->d_theta.p, c->d_psi.p, c->d_matC.p, du.p, lam.p, dg.p, s);
        g_launches += 1;
        from_device(grad, dg.p, m.n_elem, s);
    });
}

int gl_profile(gl_ctx *c, int enable) {
    return guard([&] {
        require_ctx(c);
        Prof &P = c->prof;
        if (enable && !P.on)
            for (auto &e : P.ev) GL_CUDA(cudaEventCreate(&e));
        if (!enable && P.on) {
            GL_CUDA(cudaStreamSynchronize(c->stream));
            for (auto &e : P.ev) cudaEventDestroy(e);
        }
        P.on = enable != 0;
        for (int i = 0; i < PH_N; ++i) {
            P.ms[i] = 0;
            P.count[i] = 0;
            P.pending[i] = 0;
        }
    });
}

int gl_profile_read(gl_ctx *c, gl_profile_data *out) {
    return guard([&] {
        require_ctx(c);
        GL_REQUIRE(out, "null output");
        for (int ph = 0; ph < PH_N; ++ph) prof_fold(c, ph);
        out->ms_ku = c->prof.ms[PH_KU];
        out->ms_local = c->prof.ms[PH_LOCAL];
        out->ms_coarse = c->prof.ms[PH_COARSE];
        out->n_ku = c->prof.count[PH_KU];
        out->n_local = c->prof.count[PH_LOCAL];
        out->n_coarse = c->prof.count[PH_COARSE];
        out->factor_entries = c->PD.l_size;
        out->local_dofs = c->PD.n_local;
        out->factor_bytes_per_entry = c->opts.precision == GL_PREC_MIXED ? 4 : 8;
        out->n_elem = c->m.n_elem;
        out->n_dof = c->m.n_dof;
        out->n_sub = (int)c->boxes.size();
        out->n_coarse_dim = c->n0;
        out->factor_levels = 0;
        for (auto &L : c->PD.levels)
            if (!L.fronts.empty()) ++out->factor_levels;
    });
}

long long gl_kernel_launches(void) { return g_launches.load(); }

int gl_geneo_eigenvalues(gl_ctx *c, double *lambda, int capacity, int *count) {
    return guard([&] {
        require_ctx(c);
        if (!c->ready) fail(GL_ERR_STATE, "before gl_setup");
        GL_REQUIRE(count, "null count");
        *count = (int)c->eig.size();
        if (lambda) {
            GL_REQUIRE(capacity >= (int)c->eig.size(), "capacity too small");
            std::copy(c->eig.begin(), c->eig.end(), lambda);
        }
    });
}

}  // extern "C"
