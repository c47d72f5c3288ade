// Problem-level setup shared by the single-laminate context and the batch:
// decomposition, symbolic analysis with global numbering, local element maps
// and the GenEO coarse space (Section 2.3, Fig. eig).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <mutex>
#include <thread>

#include "problem.h"

namespace gl {

namespace {

// Coarse columns whose Cholesky pivot of the unit-diagonal-scaled K_0 falls to
// 1e-10 or below (the column lies within an angle of about 1e-5, in the K
// inner product, of the span of the earlier ones) are dropped as dependent:
// this happens when two subdomains coincide (a box grown by the overlap to the
// whole extent of a narrow laminate) or when Xi_j p vanishes.
constexpr double COARSE_DROP_TOL = 1e-10;

template <class F>
void parallel_for(int n, F fn) {
    int nt = std::max(1u, std::min(std::thread::hardware_concurrency(), 32u));
    nt = std::min(nt, n);
    std::atomic<int> next(0);
    std::vector<std::thread> th;
    std::vector<Error> errs;
    std::mutex mu;
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
                }
            }
        });
    for (auto &t : th) t.join();
    if (!errs.empty()) throw errs.front();
}

std::vector<std::pair<int, int>> split_range(int n, int p) {
    std::vector<std::pair<int, int>> out;
    int q = n / p, r = n % p, s = 0;
    for (int i = 0; i < p; ++i) {
        int size = q + (i < r ? 1 : 0);
        out.push_back({s, s + size});
        s += size;
    }
    return out;
}

void check_err(const Problem &P, const char *what) {
    int h = 0;
    GL_CUDA(cudaMemcpyAsync(&h, P.d_err, sizeof(int), cudaMemcpyDeviceToHost, P.stream));
    GL_CUDA(cudaStreamSynchronize(P.stream));
    if (h) {
        GL_CUDA(cudaMemsetAsync(P.d_err, 0, sizeof(int), P.stream));
        fail(GL_ERR_NOT_SPD, std::string(what) + ": non-positive pivot");
    }
}

// G (n x m, column stride n) [gdof_j[i] - gshift, :] = Y_j[i, :] (or 0)
__global__ void k_scatter_cols(const int64_t *__restrict__ gdof, int64_t off, int64_t n, const double *__restrict__ Y,
                               int64_t yoff, int m, double *__restrict__ G, int64_t N, int64_t gshift, int zero) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n * m; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t a = i / n, r = i % n;
        G[a * N + gdof[off + r] - gshift] = zero ? 0.0 : Y[yoff + a * n + r];
    }
}

// K0[(row0 + a) + (col0 + b) * n0] = sum_i Z_l[i, a] G[gdof_l[i] - gshift, b]
__global__ void __launch_bounds__(256) k_coarse_block(const int64_t *__restrict__ gdof, int64_t off, int64_t n,
                                                      const double *__restrict__ Z, int64_t zoff, int m,
                                                      const double *__restrict__ G, int64_t N, int64_t gshift,
                                                      double *__restrict__ K0, int64_t n0, int row0, int col0) {
    const int a = blockIdx.x / m, b = blockIdx.x % m;
    double v = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) v += Z[zoff + a * n + i] * G[b * N + gdof[off + i] - gshift];
    __shared__ double red[256];
    red[threadIdx.x] = v;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) K0[(row0 + a) + (int64_t)(col0 + b) * n0] = red[0];
}

}  // namespace

void part_boxes(const MeshHost &m, int px, int py, int pz, int overlap, std::vector<SubBox> &out) {
    auto rx = split_range(m.nx, px), ry = split_range(m.ny, py), rz = split_range(m.nz, pz);
    const int ne[3] = {m.nx, m.ny, m.nz};
    for (int kz = 0; kz < pz; ++kz)
        for (int ky = 0; ky < py; ++ky)
            for (int kx = 0; kx < px; ++kx) {
                SubBox b{};
                std::pair<int, int> core[3] = {rx[kx], ry[ky], rz[kz]};
                for (int d = 0; d < 3; ++d) {
                    int lo = std::max(0, core[d].first - overlap), hi = std::min(ne[d], core[d].second + overlap);
                    b.ebox[2 * d] = lo;
                    b.ebox[2 * d + 1] = hi;
                    b.nbox[2 * d] = 2 * lo;
                    b.nbox[2 * d + 1] = 2 * hi;
                    b.art[2 * d] = lo > 0;
                    b.art[2 * d + 1] = hi < ne[d];
                }
                out.push_back(b);
            }
}

void problem_symbolic(const Problem &P, bool neumann, int leaf_nodes, std::vector<SubSymbolic> &syms) {
    const int nsub = (int)P.boxes.size();
    syms.assign(nsub, SubSymbolic());
    parallel_for(nsub, [&](int j) {
        const Part &pt = P.parts[P.sub_part[j]];
        build_symbolic(*pt.m, P.boxes[j], pt.is_dir, neumann, leaf_nodes, syms[j]);
        for (auto &g : syms[j].gdof) g += pt.dof_off;
        for (auto &e : syms[j].pair_elem) e += (int)pt.elem_off;
    });
}

void problem_local_elems(const Problem &P, int s0, int s1, const FactorPlan &plan, LocalElems &E) {
    std::vector<int> elem, sub, loc;
    for (int j = s0; j < s1; ++j) {
        const Part &pt = P.parts[P.sub_part[j]];
        const MeshHost &m = *pt.m;
        const SubBox &b = P.boxes[j];
        const int jl = j - s0;
        const int nbx = b.nbox[1] - b.nbox[0] + 1, nby = b.nbox[3] - b.nbox[2] + 1, nbz = b.nbox[5] - b.nbox[4] + 1;
        std::vector<int> map((size_t)nbx * nby * nbz * 3, -1);
        const int64_t off = plan.vec_off[jl];
        for (int64_t i = 0; i < plan.vec_len[jl]; ++i) {
            int64_t g = plan.h_gdof[off + i] - pt.dof_off;
            int64_t node = g / 3;
            int comp = (int)(g % 3);
            int x = (int)(node % m.NX), y = (int)((node / m.NX) % m.NY), z = (int)(node / ((int64_t)m.NX * m.NY));
            map[3 * ((size_t)(x - b.nbox[0]) + (size_t)nbx * ((y - b.nbox[2]) + (size_t)nby * (z - b.nbox[4]))) + comp] =
                (int)i;
        }
        for (int ez = b.ebox[4]; ez < b.ebox[5]; ++ez)
            for (int ey = b.ebox[2]; ey < b.ebox[3]; ++ey)
                for (int ex = b.ebox[0]; ex < b.ebox[1]; ++ex) {
                    elem.push_back((int)(pt.elem_off + ex + (int64_t)m.nx * (ey + (int64_t)m.ny * ez)));
                    sub.push_back(jl);
                    for (int a = 0; a < 27; ++a) {
                        int yg = 2 * ey + (a / 3) % 3;
                        if (m.periodic && yg == m.NY - 1) yg = 0;   // the first-plane partner carries the DOFs
                        int x = 2 * ex + a % 3 - b.nbox[0], y = yg - b.nbox[2], z = 2 * ez + a / 9 - b.nbox[4];
                        for (int cc = 0; cc < 3; ++cc)
                            loc.push_back(map[3 * ((size_t)x + (size_t)nbx * (y + (size_t)nby * z)) + cc]);
                    }
                }
    }
    E.n_pairs = (int64_t)elem.size();
    E.elem.upload(elem, P.stream);
    E.sub.upload(sub, P.stream);
    E.loc.upload(loc, P.stream);
    GL_CUDA(cudaStreamSynchronize(P.stream));
}

void problem_coarse(const Problem &P, const gl_opts &o, const FactorPlan &PD, int leaf_nodes, Coarse &out) {
    cudaStream_t s = P.stream;
    const int nev = o.nev;
    const double sigma = o.sigma > 0 ? o.sigma : 1e-3;
    const int nsub = (int)P.boxes.size();
    std::vector<SubSymbolic> syms;
    problem_symbolic(P, true, leaf_nodes, syms);
    build_plan(syms, out.PN, s);
    out.PN.s20 = PD.s20;
    P.stamp("Neumann symbolic");
    FactorPlan &PN = out.PN;
    for (int j = 0; j < nsub; ++j)
        if (PN.vec_len[j] < nev) fail(GL_ERR_INVALID_ARG, "subdomain has fewer DOFs than nev");
    // partition of unity: 1/multiplicity over the Dirichlet (interior) sets, 0 on artificial boundaries
    std::vector<int> mult(P.n_dof, 0);
    for (int64_t g : PD.h_gdof) mult[g] += 1;
    std::vector<double> xi(PN.n_local, 0.0);
    for (int j = 0; j < nsub; ++j) {
        const Part &pt = P.parts[P.sub_part[j]];
        const MeshHost &m = *pt.m;
        const SubBox &b = P.boxes[j];
        for (int64_t i = 0; i < PN.vec_len[j]; ++i) {
            const int64_t g = PN.h_gdof[PN.vec_off[j] + i];
            const int64_t node = (g - pt.dof_off) / 3;
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
    out.nev = nev;
    out.n0 = nsub * nev;
    out.Z.alloc(nl * nev);
    out.eig.assign((size_t)nsub * nev, 0.0);
    const int iters = o.eig_iters > 0 ? o.eig_iters : 100;
    // Groups of subdomains: factor of A^N + sigma Xi A^N Xi and block subspace
    // iteration for the largest mu of B p = mu M p, one group at a time.
    const int64_t budget = (int64_t)((o.eig_group_bytes > 0 ? o.eig_group_bytes : 4e10) / sizeof(double));
    int j0 = 0, max_its = 0;
    while (j0 < nsub) {
        int j1 = j0;
        int64_t acc = 0;
        while (j1 < nsub && (j1 == j0 || acc + syms[j1].l_size <= budget)) acc += syms[j1++].l_size;
        const int ng = j1 - j0;
        ++out.n_groups;
        std::vector<SubSymbolic> gs(syms.begin() + j0, syms.begin() + j1);
        FactorPlan PG;
        build_plan(gs, PG, s);
        PG.ws_budget_bytes = PD.ws_budget_bytes;
        PG.s20 = PD.s20;
        gs.clear();
        const int64_t goff = PN.vec_off[j0], gl = PG.n_local;
        DBuf<double> LN;
        LN.alloc(PG.l_size);
        const double *xg = d_xi.p + goff;
        numeric_factor<double>(PG, P.C, P.geo, xg, sigma, LN.p, P.d_err, s);
        check_err(P, "GenEO shifted Neumann factorisation");
        P.stamp("Neumann factorisation (group)");
        LocalElems E;
        problem_local_elems(P, j0, j1, PG, E);
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
        local_K_apply(PG, E, P.C, P.geo, xg, V.p, BV.p, k, s);            // BV = Xi A^N Xi V
        std::vector<double> mu_prev((size_t)ng * k, 0.0), mu_now((size_t)ng * k);
        // optional per-step timing of the iteration (GL_VERBOSE)
        const bool timed = std::getenv("GL_VERBOSE") != nullptr;
        cudaEvent_t ev[6] = {};
        double step_ms[5] = {0, 0, 0, 0, 0};
        if (timed)
            for (auto &e : ev) GL_CUDA(cudaEventCreate(&e));
        auto mark = [&](int i) {
            if (timed) GL_CUDA(cudaEventRecord(ev[i], s));
        };
        int it = 0;
        for (; it < iters; ++it) {
            // W = M^{-1} B V
            mark(0);
            GL_CUDA(cudaMemcpyAsync(tmp.p, BV.p, sizeof(double) * gl * k, cudaMemcpyDeviceToDevice, s));
            factor_solve<double>(PG, LN.p, tmp.p, k, s);
            std::swap(V.p, tmp.p);
            mark(1);
            BW.zero(s);
            local_K_apply(PG, E, P.C, P.geo, xg, V.p, BW.p, k, s);         // BW = B W
            mark(2);
            local_gram(PG, V.p, BV.p, k, GM.p, s);                          // W^T M W = W^T (B V)
            local_gram(PG, V.p, BW.p, k, GB.p, s);                          // W^T B W
            mark(3);
            small_geneig(ng, k, GB.p, GM.p, Y.p, mu.p, P.d_err, s);
            check_err(P, "GenEO Rayleigh-Ritz");
            mark(4);
            local_rotate(PG, V.p, Y.p, k, tmp.p, s);
            local_rotate(PG, BW.p, Y.p, k, tmp.p, s);
            mark(5);
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
            if (timed)
                for (int q = 0; q < 5; ++q) {
                    float ms = 0.f;
                    GL_CUDA(cudaEventElapsedTime(&ms, ev[q], ev[q + 1]));
                    step_ms[q] += ms;
                }
            // Ritz values settle like rate^(2 it); a change of 1e-10 leaves the Ritz vectors
            // accurate to about 1e-5, far below what changes the coarse space's effect on PCG.
            if (it >= 4 && change < 1e-10) {
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
            const double nit = std::max(it, 1);
            std::fprintf(stderr,
                         "[gl]     per iteration: solve %.1f ms, local K %.1f ms, Gram %.1f ms, Rayleigh-Ritz %.1f ms, "
                         "rotate %.1f ms (k = %d)\n",
                         step_ms[0] / nit, step_ms[1] / nit, step_ms[2] / nit, step_ms[3] / nit, step_ms[4] / nit, k);
        }
        if (timed)
            for (auto &e : ev) cudaEventDestroy(e);
        max_its = std::max(max_its, it);
        for (int j = 0; j < ng; ++j)
            for (int a = 0; a < nev; ++a) out.eig[(size_t)(j0 + j) * nev + a] = 1.0 / mu_now[(size_t)j * k + a] - sigma;
        // Z columns of these subdomains (whole-problem Neumann layout, nev columns)
        for (int j = 0; j < ng; ++j) {
            const int64_t n = PG.vec_len[j];
            GL_CUDA(cudaMemcpy2DAsync(out.Z.p + PN.vec_off[j0 + j] * nev, n * sizeof(double), V.p + PG.vec_off[j] * k,
                                      n * sizeof(double), n * sizeof(double), nev, cudaMemcpyDeviceToDevice, s));
        }
        P.stamp("GenEO subspace iteration (group)");
        j0 = j1;
    }
    out.eig_iters = max_its;
    syms.clear();
    scale_rows(PN, out.Z.p, d_xi.p, nev, s);                        // Z = Xi p
    LocalElems E;
    problem_local_elems(P, 0, nsub, PN, E);
    // K_0 = Z^T K Z per part: Y_j = A^N_j Z_j, then blocks against the overlapping subdomains of the part
    DBuf<double> KZ;
    KZ.alloc(nl * nev);
    KZ.zero(s);
    local_K_apply(PN, E, P.C, P.geo, nullptr, out.Z.p, KZ.p, nev, s);
    out.koff.clear();
    out.kvoff.clear();
    out.n_dropped = 0;
    out.part_dropped.assign(P.parts.size(), 0);
    out.kn.clear();
    int64_t ktot = 0;
    for (const Part &pt : P.parts) {
        int n0p = (pt.sub1 - pt.sub0) * nev;
        out.koff.push_back(ktot);
        out.kvoff.push_back(pt.sub0 * nev);
        out.kn.push_back(n0p);
        ktot += (int64_t)n0p * n0p;
    }
    out.Kinv.alloc(std::max<int64_t>(ktot, 1));
    for (size_t ip = 0; ip < P.parts.size(); ++ip) {
        const Part &pt = P.parts[ip];
        const int n0p = out.kn[ip];
        if (n0p == 0) continue;
        const int64_t Np = pt.m->n_dof;
        DBuf<double> G, K0;
        G.alloc((size_t)Np * nev);
        G.zero(s);
        K0.alloc((size_t)n0p * n0p);
        K0.zero(s);
        for (int j = pt.sub0; j < pt.sub1; ++j) {
            int64_t nj = PN.vec_len[j], oj = PN.vec_off[j];
            k_scatter_cols<<<256, 256, 0, s>>>(PN.d_gdof.p, oj, nj, KZ.p, oj * nev, nev, G.p, Np, pt.dof_off, 0);
            for (int l = pt.sub0; l < pt.sub1; ++l) {
                bool overlap = true;
                for (int d = 0; d < 3; ++d)
                    if (P.boxes[l].nbox[2 * d] > P.boxes[j].nbox[2 * d + 1] ||
                        P.boxes[j].nbox[2 * d] > P.boxes[l].nbox[2 * d + 1])
                        overlap = false;
                if (!overlap) continue;
                k_coarse_block<<<nev * nev, 256, 0, s>>>(PN.d_gdof.p, PN.vec_off[l], PN.vec_len[l], out.Z.p,
                                                         PN.vec_off[l] * nev, nev, G.p, Np, pt.dof_off, K0.p, n0p,
                                                         (l - pt.sub0) * nev, (j - pt.sub0) * nev);
            }
            k_scatter_cols<<<256, 256, 0, s>>>(PN.d_gdof.p, oj, nj, KZ.p, oj * nev, nev, G.p, Np, pt.dof_off, 1);
            GL_CUDA(cudaGetLastError());
        }
        out.part_dropped[ip] = dense_inverse(K0.p, n0p, out.Kinv.p + out.koff[ip], P.d_err, s, COARSE_DROP_TOL);
        out.n_dropped += out.part_dropped[ip];
        check_err(P, "coarse Cholesky");
    }
    out.d_koff.upload(out.koff, s);
    out.d_kvoff.upload(out.kvoff, s);
    out.d_kn.upload(out.kn, s);
    GL_CUDA(cudaStreamSynchronize(s));
}

void coarse_apply(const Coarse &Cs, const double *r, double *z, double *c1, double *c2, cudaStream_t s) {
    if (Cs.n0 == 0) return;
    coarse_restrict(Cs.PN, Cs.Z.p, Cs.nev, r, c1, s);
    dense_symv_blocks(Cs.Kinv.p, Cs.d_koff.p, Cs.d_kvoff.p, Cs.d_kn.p, (int)Cs.kn.size(), Cs.n0, c1, c2, s);
    coarse_prolong(Cs.PN, Cs.Z.p, Cs.nev, c2, z, s);
}

}  // namespace gl
