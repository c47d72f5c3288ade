// Batched multifrontal supernodal Cholesky and triangular solves.
//
// Section 2.3 solves each overlapping subdomain problem (zero displacement on
// the artificial boundary) with a sparse direct method.  Here every subdomain
// is ordered by geometric nested dissection (symbolic.cpp); the numeric phase
// walks the dissection trees of all subdomains together, one depth level at a
// time from the leaves up, so each launch covers every front of that depth in
// every subdomain:
//   1. zero the level's dense fronts (f x f, column-major, lower triangle);
//   2. add the element-matrix entries of the front's pivot columns;
//   3. extend-add the children's update matrices (child slot 0, then slot 1);
//   4. blocked right-looking partial Cholesky of the p pivot columns:
//      diagonal block (POTRF), panel below (TRSM), trailing lower triangle
//      (SYRK/GEMM) -- the trailing update also forms the update matrix;
//   5. copy the f x p panel into the factor array.
// After all levels the stored factor is put in partitioned-inverse form
// (k_block_inverse: inverted 32x32 diagonal blocks, rows below multiplied by
// them).  The solves walk the same levels: forward (leaves to root) and
// backward, each block step a plain product with that form.
#include <algorithm>
#include <cstdio>
#include <mutex>

#include "factor.h"
#include "q2.cuh"
#include "slaves.h"

namespace gl {

constexpr int NB = 32;        // pivot block
constexpr int TILE = 64;      // trailing-update tile

// ----------------------------------------------------------------- plan

void sweep_smem_for_plan(int max_f);

void build_plan(const std::vector<SubSymbolic> &subs, FactorPlan &P, cudaStream_t s) {
    P.n_sub = (int)subs.size();
    P.vec_off.clear();
    P.vec_len.clear();
    P.fr.clear();
    P.levels.clear();
    P.h_gdof.clear();
    std::vector<int> rows, rel, pair_elem;
    std::vector<int16_t> pair_pos;
    int64_t voff = 0, loff = 0;
    int max_depth = 0;
    for (auto &S : subs) max_depth = std::max(max_depth, S.max_depth);
    P.levels.resize(max_depth + 1);
    for (int j = 0; j < P.n_sub; ++j) {
        const SubSymbolic &S = subs[j];
        P.vec_off.push_back(voff);
        P.vec_len.push_back(S.n);
        P.h_gdof.insert(P.h_gdof.end(), S.gdof.begin(), S.gdof.end());
        int base = (int)P.fr.size();
        int64_t row_base = (int64_t)rows.size(), rel_base = (int64_t)rel.size(),
                pair_base = (int64_t)pair_elem.size();
        for (size_t i = 0; i < S.sn.size(); ++i) {
            const Supernode &sn = S.sn[i];
            FrontDesc d{};
            d.l_off = loff + sn.l_off;
            d.row_off = row_base + sn.row_off;
            d.vec_off = voff;
            d.rel_off = rel_base + sn.rel_off;
            d.pair_off = pair_base + sn.emap_off;
            d.p = sn.p;
            d.q = sn.q;
            d.n_pairs = sn.n_elem_pairs;
            d.parent = sn.parent >= 0 ? base + sn.parent : -1;
            d.sub = j;
            d.slot = 0;
            if (sn.parent >= 0) d.slot = (S.sn[sn.parent].child[1] == (int)i) ? 1 : 0;
            d.first = sn.first;
            d.vlen = S.n;
            P.fr.push_back(d);
            Level &L = P.levels[sn.depth];
            L.fronts.push_back(base + (int)i);
            if (sn.parent >= 0) L.child_slot[d.slot].push_back(base + (int)i);
        }
        rows.insert(rows.end(), S.rows.begin(), S.rows.end());
        rel.insert(rel.end(), S.rel.begin(), S.rel.end());
        pair_elem.insert(pair_elem.end(), S.pair_elem.begin(), S.pair_elem.end());
        pair_pos.insert(pair_pos.end(), S.pair_pos.begin(), S.pair_pos.end());
        voff += S.n;
        loff += S.l_size;
    }
    P.n_local = voff;
    P.l_size = loff;
    P.nnz = 0;
    for (const FrontDesc &d : P.fr) P.nnz += (int64_t)d.p * (d.p + 1) / 2 + (int64_t)d.p * d.q;
    P.ws_max = 0;
    P.max_f = 0;
    for (auto &L : P.levels) {
        int64_t off = 0;
        for (int g : L.fronts) {
            FrontDesc &d = P.fr[g];
            int f = d.p + d.q;
            d.front_off = off;
            off += (int64_t)f * f;
            L.max_p = std::max(L.max_p, d.p);
            L.max_f = std::max(L.max_f, f);
        }
        L.ws = off;
        P.ws_max = std::max(P.ws_max, off);
        P.max_f = std::max(P.max_f, L.max_f);
        std::vector<int> v(L.fronts);
        L.d_fronts.upload(v, s);
        L.d_child[0].upload(L.child_slot[0], s);
        L.d_child[1].upload(L.child_slot[1], s);
    }
    // the first half of the subdomains: fronts are listed per level in subdomain order
    P.half_fronts.assign(P.levels.size(), 0);
    for (size_t d = 0; d < P.levels.size(); ++d)
        for (int g : P.levels[d].fronts)
            if (P.fr[g].sub < P.n_sub / 2) ++P.half_fronts[d];
    P.d_fr.upload(P.fr, s);
    P.d_rows.upload(rows, s);
    P.d_rel.upload(rel, s);
    P.d_pair_elem.upload(pair_elem, s);
    P.d_pair_pos.upload(pair_pos, s);
    P.d_gdof.upload(P.h_gdof, s);
    P.d_vec_off.upload(P.vec_off, s);
    P.d_vec_len.upload(P.vec_len, s);
    sweep_smem_for_plan(P.max_f);
    GL_CUDA(cudaStreamSynchronize(s));
}

// ----------------------------------------------------------------- numeric kernels

// One block per (front, element): the element stiffness
// K_e = sum_q w_q |J_q| B_q^T C_e B_q (FP64) is formed in shared memory, then
// the entries of the front's pivot columns are added into the front.  With
// sigma != 0 the entry (i, j) is scaled by 1 + sigma xi_i xi_j (the matrix
// A^N + sigma Xi A^N Xi of the GenEO pencil).
template <class T>
__global__ void __launch_bounds__(256) k_assemble(const int *__restrict__ fronts, const FrontDesc *__restrict__ D,
                                                  const int *__restrict__ pair_elem,
                                                  const int16_t *__restrict__ pair_pos, const int *__restrict__ rows,
                                                  const double *__restrict__ C, const double *__restrict__ geo,
                                                  const double *__restrict__ xi, double sigma, int s20,
                                                  T *__restrict__ ws) {
    const FrontDesc d = D[fronts[blockIdx.x]];
    const int pr_i = blockIdx.y;
    if (pr_i >= d.n_pairs) return;
    extern __shared__ double sK[];   // 81 x 81
    __shared__ int16_t sp[81];
    __shared__ double sx[81];
    __shared__ double sG[27][3];
    __shared__ double sCB[6][81];
    __shared__ double sC[36];
    __shared__ double sw;
    const int f = d.p + d.q;
    const int64_t e = pair_elem[d.pair_off + pr_i];
    const int16_t *pos = pair_pos + (d.pair_off + pr_i) * 81;
    if (threadIdx.x < 81) {
        int16_t v = pos[threadIdx.x];
        sp[threadIdx.x] = v;
        sx[threadIdx.x] = (xi && v >= 0) ? xi[d.vec_off + rows[d.row_off + v]] : 0.0;
    }
    if (threadIdx.x < 36) sC[threadIdx.x] = C[36 * e + threadIdx.x];
    Q2Tables Tb;
    Tb.init();
    double acc[26];
#pragma unroll
    for (int i = 0; i < 26; ++i) acc[i] = 0.0;
    for (int q = 0; q < 27; ++q) {
        __syncthreads();
        const int qx = q % 3, qy = (q / 3) % 3, qz = q / 9;
        const double *g = geo + 10 * (e * 27 + q);
        if (threadIdx.x < 27) {
            int a = threadIdx.x, i = a % 3, j = (a / 3) % 3, k = a / 9;
            double r0 = Tb.D[qx][i] * Tb.N[qy][j] * Tb.N[qz][k];
            double r1 = Tb.N[qx][i] * Tb.D[qy][j] * Tb.N[qz][k];
            double r2 = Tb.N[qx][i] * Tb.N[qy][j] * Tb.D[qz][k];
            for (int dd = 0; dd < 3; ++dd) sG[a][dd] = r0 * g[0 + dd] + r1 * g[3 + dd] + r2 * g[6 + dd];
        }
        if (threadIdx.x == 0) sw = g[9];
        __syncthreads();
        for (int idx = threadIdx.x; idx < 6 * 81; idx += blockDim.x) {
            int I = idx / 81, col = idx % 81, a = col / 3, c = col % 3;
            double gx = sG[a][0], gy = sG[a][1], gz = sG[a][2], v;
            if (c == 0) v = sC[6 * I + 0] * gx + sC[6 * I + 4] * gz + sC[6 * I + 5] * gy;
            else if (c == 1) v = sC[6 * I + 1] * gy + sC[6 * I + 3] * gz + sC[6 * I + 5] * gx;
            else v = sC[6 * I + 2] * gz + sC[6 * I + 3] * gy + sC[6 * I + 4] * gx;
            sCB[I][col] = v;
        }
        __syncthreads();
        const double w = sw;
        int slot = 0;
        for (int idx = threadIdx.x; idx < 6561; idx += blockDim.x, ++slot) {
            int r = idx / 81, col = idx % 81, a = r / 3, c = r % 3;
            double gx = sG[a][0], gy = sG[a][1], gz = sG[a][2], v;
            if (c == 0) v = gx * sCB[0][col] + gz * sCB[4][col] + gy * sCB[5][col];
            else if (c == 1) v = gy * sCB[1][col] + gz * sCB[3][col] + gx * sCB[5][col];
            else v = gz * sCB[2][col] + gy * sCB[3][col] + gx * sCB[4][col];
            acc[slot] += w * v;
        }
    }
    {
        int slot = 0;
        for (int idx = threadIdx.x; idx < 6561; idx += blockDim.x, ++slot) sK[idx] = acc[slot];
    }
    __syncthreads();
    if (s20) {
        // serendipity element: K <- P^T K P, P the identity on the 20 nodes and the fixed
        // combinations of them on the 7 face/body centres; first the columns, then the rows
        // (only master rows and columns are updated; the slaves' are never assembled)
        for (int idx = threadIdx.x; idx < 6561; idx += blockDim.x) {
            const int r = idx / 81, col = idx % 81, a = col / 3, cc = col % 3;
            if (s20_is_slave(a)) continue;
            double v = sK[idx];
            for (int b = 0; b < 27; ++b)
                if (s20_is_slave(b)) {
                    const double w = s20_weight(b, a);
                    if (w != 0.0) v += w * sK[81 * r + 3 * b + cc];
                }
            sK[idx] = v;
        }
        __syncthreads();
        for (int idx = threadIdx.x; idx < 6561; idx += blockDim.x) {
            const int r = idx / 81, col = idx % 81, a = r / 3, cc = r % 3;
            if (s20_is_slave(a) || s20_is_slave(col / 3)) continue;
            double v = sK[idx];
            for (int b = 0; b < 27; ++b)
                if (s20_is_slave(b)) {
                    const double w = s20_weight(b, a);
                    if (w != 0.0) v += w * sK[81 * (3 * b + cc) + col];
                }
            sK[idx] = v;
        }
        __syncthreads();
    }
    T *F = ws + d.front_off;
    for (int idx = threadIdx.x; idx < 6561; idx += blockDim.x) {
        int c = idx / 81, r = idx % 81;    // column (pivot) c, row r
        int pc = sp[c], pr = sp[r];
        if (pc < 0 || pc >= d.p || pr < pc) continue;
        double v = sK[81 * r + c];
        if (sigma != 0.0) v *= 1.0 + sigma * sx[r] * sx[c];
        atomicAdd(F + pr + (int64_t)pc * f, (T)v);
    }
}

template <class T>
__global__ void k_extend_add(const int *__restrict__ children, const FrontDesc *__restrict__ D,
                             const int *__restrict__ rel, const T *__restrict__ ws_child, T *__restrict__ ws_par) {
    const FrontDesc c = D[children[blockIdx.x]];
    const int qc = c.q;
    if (qc == 0) return;
    const FrontDesc par = D[c.parent];
    const int fc = c.p + c.q, fp = par.p + par.q;
    const int *rm = rel + c.rel_off;
    const T *U = ws_child + c.front_off;
    T *F = ws_par + par.front_off;
    for (int j = blockIdx.y; j < qc; j += gridDim.y) {
        const int pj = rm[j];
        const T *Uc = U + (int64_t)(c.p + j) * fc + c.p;
        T *Fc = F + (int64_t)pj * fp;
        for (int i = j + threadIdx.x; i < qc; i += blockDim.x) Fc[rm[i]] += Uc[i];
    }
}

// Diagonal block Cholesky (kb <= 32) of each front at pivot offset k0.
template <class T>
__global__ void k_potrf(const int *__restrict__ fronts, const FrontDesc *__restrict__ D, T *__restrict__ ws, int k0,
                        int *__restrict__ err, T drop, int *__restrict__ drops) {
    const FrontDesc d = D[fronts[blockIdx.x]];
    if (k0 >= d.p) return;
    const int kb = min(NB, d.p - k0), f = d.p + d.q;
    T *A = ws + d.front_off + k0 + (int64_t)k0 * f;
    __shared__ T a[NB][NB + 1];
    for (int idx = threadIdx.x; idx < kb * kb; idx += blockDim.x) {
        int i = idx % kb, j = idx / kb;
        a[i][j] = i >= j ? A[i + (int64_t)j * f] : T(0);
    }
    __syncthreads();
    for (int j = 0; j < kb; ++j) {
        if (threadIdx.x == 0) {
            T v = a[j][j];
            if (drop > T(0) && fabs(v) <= drop) {
                // dependent column (drop mode): zero pivot, the column leaves the factor
                atomicAdd(drops, 1);
                a[j][j] = T(0);
            } else {
                if (!(v > T(0))) {
                    atomicExch(err, 1);
                    v = T(1);
                }
                a[j][j] = sqrt(v);
            }
        }
        __syncthreads();
        T djj = a[j][j];
        for (int i = j + 1 + threadIdx.x; i < kb; i += blockDim.x) a[i][j] = djj != T(0) ? a[i][j] / djj : T(0);
        __syncthreads();
        for (int idx = threadIdx.x; idx < kb * kb; idx += blockDim.x) {
            int i = idx % kb, k = idx / kb;
            if (k > j && i >= k) a[i][k] -= a[i][j] * a[k][j];
        }
        __syncthreads();
    }
    for (int idx = threadIdx.x; idx < kb * kb; idx += blockDim.x) {
        int i = idx % kb, j = idx / kb;
        if (i >= j) A[i + (int64_t)j * f] = a[i][j];
    }
}

// Panel below the diagonal block: rows r in [k0+kb, f) <- row * L_kk^{-T}.
template <class T>
__global__ void k_trsm(const int *__restrict__ fronts, const FrontDesc *__restrict__ D, T *__restrict__ ws, int k0) {
    const FrontDesc d = D[fronts[blockIdx.x]];
    if (k0 >= d.p) return;
    const int kb = min(NB, d.p - k0), f = d.p + d.q;
    const int r = k0 + kb + blockIdx.y * blockDim.x + threadIdx.x;
    __shared__ T l[NB][NB + 1];
    T *F = ws + d.front_off;
    for (int idx = threadIdx.x; idx < kb * kb; idx += blockDim.x) {
        int i = idx % kb, j = idx / kb;
        l[i][j] = i >= j ? F[(k0 + i) + (int64_t)(k0 + j) * f] : T(0);
    }
    __syncthreads();
    if (r >= f) return;
    T x[NB];
#pragma unroll
    for (int j = 0; j < NB; ++j)
        if (j < kb) x[j] = F[r + (int64_t)(k0 + j) * f];
#pragma unroll
    for (int j = 0; j < NB; ++j) {
        if (j < kb) {
            T v = x[j];
#pragma unroll
            for (int i = 0; i < NB; ++i)
                if (i < j) v -= x[i] * l[j][i];
            x[j] = l[j][j] != T(0) ? v / l[j][j] : T(0);   // zero pivot: a dropped column
        }
    }
#pragma unroll
    for (int j = 0; j < NB; ++j)
        if (j < kb) F[r + (int64_t)(k0 + j) * f] = x[j];
}

// Trailing update of the lower triangle: F[r, c] -= sum_j P[r, j] P[c, j] for
// r >= c >= k0+kb, P the panel columns k0..k0+kb.  64x64 tiles, 256 threads.
// With cend > 0 only the columns c < min(cend, p) are updated (the rest of an
// outer panel whose trailing matrix is updated separately): the tiles are
// then those of the first column tiles of the trailing lower triangle.
template <class T>
__global__ void __launch_bounds__(256) k_syrk(const int *__restrict__ fronts, const FrontDesc *__restrict__ D,
                                              T *__restrict__ ws, int k0, int cend) {
    const FrontDesc d = D[fronts[blockIdx.x]];
    if (k0 >= d.p) return;
    const int kb = min(NB, d.p - k0), f = d.p + d.q;
    const int base = k0 + kb, m = f - base;
    if (m <= 0) return;
    const int nt = (m + TILE - 1) / TILE;
    int t = blockIdx.y, ti, tj;
    if (cend > 0) {
        const int cw = min(cend, d.p) - base;       // columns to update
        if (cw <= 0) return;
        const int ncw = (cw + TILE - 1) / TILE;
        // t -> (ti, tj), column-major over the tiles of the first ncw tile columns
        tj = 0;
        while (tj < ncw && t >= nt - tj) t -= nt - tj++;
        if (tj >= ncw) return;
        ti = tj + t;
    } else {
        if (t >= nt * (nt + 1) / 2) return;
        // t -> (ti, tj), ti >= tj, row-major over the lower triangle of tiles
        ti = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
        while ((ti + 1) * (ti + 2) / 2 <= t) ++ti;
        while (ti * (ti + 1) / 2 > t) --ti;
        tj = t - ti * (ti + 1) / 2;
    }
    const int cmax = cend > 0 ? min(cend, d.p) : f;   // columns c < cmax are updated
    const int r0 = base + ti * TILE, c0 = base + tj * TILE;
    T *F = ws + d.front_off;
    __shared__ T sa[NB][TILE + 1], sb[NB][TILE + 1];
    for (int idx = threadIdx.x; idx < NB * TILE; idx += blockDim.x) {
        int i = idx % TILE, j = idx / TILE;
        int r = r0 + i, c = c0 + i;
        sa[j][i] = (j < kb && r < f) ? F[r + (int64_t)(k0 + j) * f] : T(0);
        sb[j][i] = (j < kb && c < f) ? F[c + (int64_t)(k0 + j) * f] : T(0);
    }
    __syncthreads();
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    T acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
#pragma unroll 8
    for (int j = 0; j < NB; ++j) {
        T av[4], bv[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) av[a] = sa[j][tx + 16 * a];
#pragma unroll
        for (int b = 0; b < 4; ++b) bv[b] = sb[j][ty + 16 * b];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[a][b] += av[a] * bv[b];
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            int r = r0 + tx + 16 * a, c = c0 + ty + 16 * b;
            if (r < f && c < cmax && r >= c) F[r + (int64_t)c * f] -= acc[a][b];
        }
}

template <class T>
__global__ void k_copy_panel(const int *__restrict__ fronts, const FrontDesc *__restrict__ D,
                             const T *__restrict__ ws, T *__restrict__ L) {
    const FrontDesc d = D[fronts[blockIdx.x]];
    const int f = d.p + d.q;
    const int64_t n = (int64_t)f * d.p;
    const T *F = ws + d.front_off;
    T *out = L + d.l_off;
    for (int64_t idx = blockIdx.y * (int64_t)blockDim.x + threadIdx.x; idx < n; idx += (int64_t)gridDim.y * blockDim.x) {
        int64_t j = idx / f, i = idx % f;
        out[idx] = i >= j ? F[i + j * f] : T(0);
    }
}

// Blocked right-looking partial Cholesky of the p pivot columns of every front
// of a level.  FP64 (and FP32 with tc = false): blocks of NB = 32 pivots, each
// followed by the rank-32 update of the whole trailing lower triangle.  FP32
// with tc: outer panels of 128 columns factored with the same 32-wide steps,
// whose updates stay inside the panel, and one rank-128 update of the trailing
// matrix per panel on the tensor cores (syrk_tc.cu) -- four times the flops
// per byte of trailing matrix read and written.
static void partial_cholesky_level(const int *d_fronts, int n_fronts, const FrontDesc *d_fr, int max_p, int max_f,
                                   void *ws, bool fp32, int *d_err, cudaStream_t s, double drop = 0.0,
                                   int *d_drops = nullptr, bool tc = false) {
    if (fp32 && tc) {
        const int PW = syrk_tc_panel();
        for (int k0 = 0; k0 < max_p; k0 += PW) {
            const int kend = k0 + PW;
            for (int k1 = k0; k1 < std::min(kend, max_p); k1 += NB) {
                const int rows = std::max(1, max_f - k1);
                const int m = max_f - k1;
                const int nt = m > 0 ? (m + TILE - 1) / TILE : 0;
                const int ncw = std::min(nt, (kend - k1 - 1) / TILE + 1);    // column tiles inside the panel
                const int tiles = std::max(1, ncw * nt - ncw * (ncw - 1) / 2);
                k_potrf<float><<<n_fronts, 128, 0, s>>>(d_fronts, d_fr, (float *)ws, k1, d_err, (float)drop, d_drops);
                k_trsm<float><<<dim3(n_fronts, (rows + 127) / 128), 128, 0, s>>>(d_fronts, d_fr, (float *)ws, k1);
                k_syrk<float><<<dim3(n_fronts, tiles), 256, 0, s>>>(d_fronts, d_fr, (float *)ws, k1, kend);
                GL_CUDA(cudaGetLastError());
            }
            syrk_tc_level(d_fronts, n_fronts, d_fr, k0, max_f, (float *)ws, d_err, s);
        }
        return;
    }
    for (int k0 = 0; k0 < max_p; k0 += NB) {
        // upper bounds over the level's fronts (a front's last pivot block may be short)
        int rows = std::max(1, max_f - k0);
        int m = max_f - k0;
        int nt = m > 0 ? (m + TILE - 1) / TILE : 0;
        int tiles = std::max(1, nt * (nt + 1) / 2);
        dim3 gt(n_fronts, (rows + 127) / 128), gs(n_fronts, tiles);
        if (fp32) {
            k_potrf<float><<<n_fronts, 128, 0, s>>>(d_fronts, d_fr, (float *)ws, k0, d_err, (float)drop, d_drops);
            k_trsm<float><<<gt, 128, 0, s>>>(d_fronts, d_fr, (float *)ws, k0);
            k_syrk<float><<<gs, 256, 0, s>>>(d_fronts, d_fr, (float *)ws, k0, 0);
        } else {
            k_potrf<double><<<n_fronts, 128, 0, s>>>(d_fronts, d_fr, (double *)ws, k0, d_err, drop, d_drops);
            k_trsm<double><<<gt, 128, 0, s>>>(d_fronts, d_fr, (double *)ws, k0);
            k_syrk<double><<<gs, 256, 0, s>>>(d_fronts, d_fr, (double *)ws, k0, 0);
        }
        GL_CUDA(cudaGetLastError());
    }
}

// Partitioned-inverse form of the stored factor, used by the sweeps.  For
// every block B of 32 consecutive pivots of a front (the last one may be
// shorter): L[B,B] <- L[B,B]^{-1} (lower triangular) and, for every row i
// below B in the front (later pivots and structure rows),
// L[i,B] <- W[i,B] = L[i,B] L[B,B]^{-1}.  A forward step is then
// y_B = L[B,B]^{-1} x_B and x_i -= W[i,B] x_B, a backward step
// x_B = L[B,B]^{-T} y_B - W[i,B]^T x_i: plain products with no serial
// triangular solve.  Computed in FP64 whatever the storage type.  One CTA per
// (front, block); blocks are independent of one another.
template <class T>
__global__ void __launch_bounds__(256) k_block_inverse(const FrontDesc *__restrict__ D, T *__restrict__ L) {
    const FrontDesc d = D[blockIdx.x];
    const int jb = blockIdx.y * 32;
    if (jb >= d.p) return;
    const int kb = min(32, d.p - jb), f = d.p + d.q;
    T *Lp = L + d.l_off;
    __shared__ double Dk[32][33], Li[32][33];
    for (int idx = threadIdx.x; idx < 1024; idx += blockDim.x) {
        const int i = idx & 31, j = idx >> 5;
        Dk[i][j] = (i < kb && j < kb && i >= j) ? (double)Lp[(jb + i) + (int64_t)(jb + j) * f] : 0.0;
        Li[i][j] = 0.0;
    }
    __syncthreads();
    if (threadIdx.x < kb) {
        // column j of the inverse by forward substitution on e_j
        const int j = threadIdx.x;
        Li[j][j] = 1.0 / Dk[j][j];
        for (int i = j + 1; i < kb; ++i) {
            double acc = 0.0;
            for (int k = j; k < i; ++k) acc += Dk[i][k] * Li[k][j];
            Li[i][j] = -acc / Dk[i][i];
        }
    }
    __syncthreads();
    for (int i = jb + kb + threadIdx.x; i < f; i += blockDim.x) {
        double r[32];
#pragma unroll
        for (int k = 0; k < 32; ++k) r[k] = k < kb ? (double)Lp[i + (int64_t)(jb + k) * f] : 0.0;
#pragma unroll 1
        for (int j = 0; j < kb; ++j) {
            double w = 0.0;   // Li is lower triangular: the terms k < j vanish
#pragma unroll
            for (int k = 0; k < 32; ++k) w += r[k] * Li[k][j];
            Lp[i + (int64_t)(jb + j) * f] = (T)w;
        }
    }
    for (int idx = threadIdx.x; idx < 1024; idx += blockDim.x) {
        const int i = idx & 31, j = idx >> 5;
        if (i < kb && j < kb && i >= j) Lp[(jb + i) + (int64_t)(jb + j) * f] = (T)Li[i][j];
    }
}

// Subdomains are factorised in consecutive groups whose two live levels of
// dense fronts fit a workspace budget; inside a group every level is one set
// of batched launches.
template <class T>
void numeric_factor(FactorPlan &P, const double *C, const double *geo, const double *xi, double sigma, T *L,
                    int *d_err, cudaStream_t s) {
    static SmemLimit assemble_smem;
    raise_smem_limit(assemble_smem, 6561 * 8, [](size_t v) {
        GL_CUDA(cudaFuncSetAttribute(k_assemble<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)v));
    });
    const int nlev = (int)P.levels.size();
    const int64_t budget = (int64_t)(P.ws_budget_bytes / sizeof(T));   // entries per workspace buffer
    std::vector<int> depth_of(P.fr.size());
    for (int d = 0; d < nlev; ++d)
        for (int g : P.levels[d].fronts) depth_of[g] = d;
    std::vector<int64_t> sub_ws((size_t)P.n_sub * nlev, 0);
    for (size_t g = 0; g < P.fr.size(); ++g) {
        int64_t f = P.fr[g].p + P.fr[g].q;
        sub_ws[(size_t)P.fr[g].sub * nlev + depth_of[g]] += f * f;
    }
    std::vector<int> first_front(P.n_sub + 1, 0);
    for (size_t g = 0; g < P.fr.size(); ++g) first_front[P.fr[g].sub + 1] = (int)g + 1;
    for (int j = 1; j <= P.n_sub; ++j) first_front[j] = std::max(first_front[j], first_front[j - 1]);
    std::vector<FrontDesc> fr = P.fr;
    DBuf<FrontDesc> d_fr;
    DBuf<T> ws[2];
    int j0 = 0;
    P.last_groups = 0;
    while (j0 < P.n_sub) {
        ++P.last_groups;
        // grow the group while every level's total stays within the budget
        std::vector<int64_t> tot(nlev, 0);
        int j1 = j0;
        while (j1 < P.n_sub) {
            bool ok = true;
            for (int d = 0; d < nlev; ++d)
                if (tot[d] + sub_ws[(size_t)j1 * nlev + d] > budget) ok = false;
            if (!ok && j1 > j0) break;
            for (int d = 0; d < nlev; ++d) tot[d] += sub_ws[(size_t)j1 * nlev + d];
            ++j1;
        }
        // per-level lists of this group's fronts and their workspace offsets
        std::vector<std::vector<int>> lev(nlev), child[2];
        child[0].resize(nlev);
        child[1].resize(nlev);
        std::vector<int> max_p(nlev, 0), max_f(nlev, 0), max_pairs(nlev, 0);
        std::vector<int64_t> lev_ws(nlev, 0), max_panel(nlev, 0);
        for (int g = first_front[j0]; g < first_front[j1]; ++g) {
            int d = depth_of[g];
            int f = fr[g].p + fr[g].q;
            fr[g].front_off = lev_ws[d];
            lev_ws[d] += (int64_t)f * f;
            lev[d].push_back(g);
            if (fr[g].parent >= 0) child[fr[g].slot][d].push_back(g);
            max_p[d] = std::max(max_p[d], fr[g].p);
            max_f[d] = std::max(max_f[d], f);
            max_pairs[d] = std::max(max_pairs[d], fr[g].n_pairs);
            max_panel[d] = std::max<int64_t>(max_panel[d], (int64_t)f * fr[g].p);
        }
        int64_t need = 1;
        for (int d = 0; d < nlev; ++d) need = std::max(need, lev_ws[d]);
        if ((int64_t)ws[0].n < need) {
            ws[0].alloc(need);
            ws[1].alloc(need);
        }
        d_fr.upload(fr, s);
        std::vector<DBuf<int>> d_lev(nlev), d_ch0(nlev), d_ch1(nlev);
        for (int d = 0; d < nlev; ++d) {
            d_lev[d].upload(lev[d], s);
            d_ch0[d].upload(child[0][d], s);
            d_ch1[d].upload(child[1][d], s);
        }
        for (int dpt = nlev - 1; dpt >= 0; --dpt) {
            const int nf = (int)lev[dpt].size();
            if (nf == 0) continue;
            T *W = ws[dpt & 1].p;
            GL_CUDA(cudaMemsetAsync(W, 0, lev_ws[dpt] * sizeof(T), s));
            if (max_pairs[dpt] > 0) {
                k_assemble<T><<<dim3(nf, max_pairs[dpt]), 256, 6561 * 8, s>>>(
                    d_lev[dpt].p, d_fr.p, P.d_pair_elem.p, P.d_pair_pos.p, P.d_rows.p, C, geo, xi, sigma, P.s20 ? 1 : 0,
                    W);
                GL_CUDA(cudaGetLastError());
            }
            if (dpt + 1 < nlev) {
                for (int slot = 0; slot < 2; ++slot) {
                    int nc = (int)child[slot][dpt + 1].size();
                    if (!nc) continue;
                    int ycols = std::min(std::max(1, max_f[dpt + 1] / 8), 1024);
                    k_extend_add<T><<<dim3(nc, ycols), 128, 0, s>>>(slot ? d_ch1[dpt + 1].p : d_ch0[dpt + 1].p,
                                                                  d_fr.p, P.d_rel.p, ws[(dpt + 1) & 1].p, W);
                    GL_CUDA(cudaGetLastError());
                }
            }
            partial_cholesky_level(d_lev[dpt].p, nf, d_fr.p, max_p[dpt], max_f[dpt], W, sizeof(T) == 4, d_err, s,
                                   0.0, nullptr, sizeof(T) == 4 && P.tc_update);
            int gy = (int)std::min<int64_t>(std::max<int64_t>(1, (max_panel[dpt] + 255) / 256), 4096);
            k_copy_panel<T><<<dim3(nf, gy), 256, 0, s>>>(d_lev[dpt].p, d_fr.p, W, L);
            GL_CUDA(cudaGetLastError());
        }
        GL_CUDA(cudaStreamSynchronize(s));   // the group's lists are released at the end of this scope
        j0 = j1;
    }
    int max_p = 0;
    for (const FrontDesc &d : P.fr) max_p = std::max(max_p, d.p);
    if (!P.fr.empty() && max_p > 0) {
        k_block_inverse<T><<<dim3((unsigned)P.fr.size(), (max_p + 31) / 32), 256, 0, s>>>(P.d_fr.p, L);
        GL_CUDA(cudaGetLastError());
        GL_CUDA(cudaStreamSynchronize(s));
    }
}

template void numeric_factor<double>(FactorPlan &, const double *, const double *, const double *, double, double *,
                                     int *, cudaStream_t);
template void numeric_factor<float>(FactorPlan &, const double *, const double *, const double *, double, float *,
                                    int *, cudaStream_t);

// ----------------------------------------------------------------- solves

// Threads per CTA of the sweeps: 256, or 512 on levels with fewer fronts than
// eight per SM (the upper dissection levels, large fronts), where one CTA per
// front would otherwise leave most warp slots empty.  Both kernels loop
// over rows and columns with the block size, so either works.
constexpr int SWEEP_MAX_THREADS = 512;
constexpr int SWEEP_WIDE_BELOW = 1216;  // fronts per level
// Threads per CTA of the sweeps on levels with at least SWEEP_WIDE_BELOW fronts
// (SMALL: those whose largest front has at most SWEEP_SMALL_F rows).
#ifndef GL_SWEEP_FWD_THREADS
#define GL_SWEEP_FWD_THREADS 256
#endif
#ifndef GL_SWEEP_BWD_THREADS
#define GL_SWEEP_BWD_THREADS 256
#endif
#ifndef GL_SWEEP_FWD_SMALL_THREADS
#define GL_SWEEP_FWD_SMALL_THREADS 256
#endif
#ifndef GL_SWEEP_BWD_SMALL_THREADS
#define GL_SWEEP_BWD_SMALL_THREADS 128
#endif
#ifndef GL_SWEEP_SMALL_F
#define GL_SWEEP_SMALL_F 800
#endif
// Threads per CTA of the sweeps on levels with fewer than SWEEP_WIDE_BELOW fronts.
#ifndef GL_SWEEP_FWD_WIDE_THREADS
#define GL_SWEEP_FWD_WIDE_THREADS 512
#endif
#ifndef GL_SWEEP_BWD_WIDE_THREADS
#define GL_SWEEP_BWD_WIDE_THREADS 512
#endif

// The forward sweep of FP64 (FP32) factors treats the structure rows after the
// triangle when GL_FWD_SPLIT64 (GL_FWD_SPLIT32) is 1, block by block otherwise.
#ifndef GL_FWD_SPLIT64
#define GL_FWD_SPLIT64 0
#endif
#ifndef GL_FWD_SPLIT32
#define GL_FWD_SPLIT32 1
#endif
template <class T>
constexpr bool fwd_split() {
    return sizeof(T) == 8 ? GL_FWD_SPLIT64 != 0 : GL_FWD_SPLIT32 != 0;
}

// The sweeps read the partitioned-inverse form written by k_block_inverse.
// Dynamic shared memory of both starts with the front's dense vector v
// (f x NR entries).
//
// Forward substitution for the fronts of one level, one CTA per front.  The
// panel of a front is its pivot rows (the triangle, in partitioned-inverse
// form) over its structure rows (a q x p rectangle).
//   1. the triangle, block by block: x_B (the pivot values as left by the
//      earlier blocks) is kept in X; the block's own rows hold
//      L[B,B]^{-1} (zero above the diagonal), so they get y_B = L[B,B]^{-1} x_B,
//      and the later pivot rows x_i -= W[i,B] x_B -- one row per thread, the
//      block's rows one more row group.
//   2. the rectangle at once: structure row i gets -sum_c W[i, c] X_c over all
//      pivot columns c, one row per thread with no block barrier, and is added
//      into the ancestors' entries atomically (siblings share rows).
// One FMA per stored entry; no serial triangular solve remains.
template <class T, int NR>
__device__ __forceinline__ void fwd_row(const T *__restrict__ col0, int64_t ld, int i, int kb, const T *xb, int xs,
                                        T acc[NR]) {
    // acc[r] = sum over the kb columns of the block at col0 of W[i, j] xb[j + r xs]
    if (kb == 32 && NR == 1) {
        T l[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) l[j] = col0[i + (int64_t)j * ld];
        T a0 = T(0), a1 = T(0);
#pragma unroll
        for (int j = 0; j < 32; j += 2) {
            a0 += l[j] * xb[j];
            a1 += l[j + 1] * xb[j + 1];
        }
        acc[0] = a0 + a1;
    } else if (kb == 32) {
        // several right-hand sides: the row's loads in four groups of eight
#pragma unroll
        for (int r = 0; r < NR; ++r) acc[r] = T(0);
#pragma unroll
        for (int jc = 0; jc < 32; jc += 8) {
            T l[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) l[j] = col0[i + (int64_t)(jc + j) * ld];
#pragma unroll
            for (int r = 0; r < NR; ++r)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[r] += l[j] * xb[jc + j + r * xs];
        }
    } else {
#pragma unroll
        for (int r = 0; r < NR; ++r) acc[r] = T(0);
        for (int j = 0; j < kb; ++j) {
            const T l = col0[i + (int64_t)j * ld];
#pragma unroll
            for (int r = 0; r < NR; ++r) acc[r] += l * xb[j + r * xs];
        }
    }
}

template <class T, int NR, bool SPLIT>
__global__ void __launch_bounds__(SWEEP_MAX_THREADS) k_fwd(const int *__restrict__ fronts, const FrontDesc *__restrict__ D,
                                             const T *__restrict__ L, const int *__restrict__ rows, T *__restrict__ x,
                                             int kcols, int c0) {
    extern __shared__ unsigned char smraw[];
    const FrontDesc d = D[fronts[blockIdx.x]];
    const int p = d.p, f = d.p + d.q, n = d.vlen;
    T *v = reinterpret_cast<T *>(smraw);   // the front's vector, f x NR
    T *X = v + (int64_t)f * NR;             // x_B of every block, p x NR
    T *xs = x + d.vec_off * kcols + (int64_t)c0 * n;
    // rows updated block by block: the pivot rows only (SPLIT), or the structure rows too
    const int rend = SPLIT ? p : f;
    for (int i = threadIdx.x; i < rend; i += blockDim.x)
#pragma unroll
        for (int r = 0; r < NR; ++r) v[i + r * f] = i < p ? xs[(int64_t)r * n + d.first + i] : T(0);
    __syncthreads();
    const T *Lp = L + d.l_off;
    // 1. the triangle (and, unless SPLIT, the rectangle block by block)
    for (int jb = 0; jb < p; jb += 32) {
        const int kb = min(32, p - jb);
        if (threadIdx.x < 32 * NR) {
            const int j = threadIdx.x & 31, r = threadIdx.x >> 5;
            if (j < kb) X[jb + j + r * p] = v[jb + j + r * f];
        }
        __syncthreads();
        for (int i = jb + threadIdx.x; i < rend; i += blockDim.x) {
            T acc[NR];
            fwd_row<T, NR>(Lp + (int64_t)jb * f, f, i, kb, X + jb, p, acc);
            if (i < jb + kb) {
#pragma unroll
                for (int r = 0; r < NR; ++r) v[i + r * f] = acc[r];
            } else {
#pragma unroll
                for (int r = 0; r < NR; ++r) v[i + r * f] -= acc[r];
            }
        }
        __syncthreads();
    }
    for (int i = threadIdx.x; i < p; i += blockDim.x)
#pragma unroll
        for (int r = 0; r < NR; ++r) xs[(int64_t)r * n + d.first + i] = v[i + r * f];
    if constexpr (!SPLIT) {
        for (int i = p + threadIdx.x; i < f; i += blockDim.x)
#pragma unroll
            for (int r = 0; r < NR; ++r) atomicAdd(xs + (int64_t)r * n + rows[d.row_off + i], v[i + r * f]);
    } else {
        // 2. the rectangle
        for (int i = p + threadIdx.x; i < f; i += blockDim.x) {
            T sum[NR];
#pragma unroll
            for (int r = 0; r < NR; ++r) sum[r] = T(0);
            for (int jb = 0; jb < p; jb += 32) {
                T acc[NR];
                fwd_row<T, NR>(Lp + (int64_t)jb * f, f, i, min(32, p - jb), X + jb, p, acc);
#pragma unroll
                for (int r = 0; r < NR; ++r) sum[r] += acc[r];
            }
            const int gi = rows[d.row_off + i];
#pragma unroll
            for (int r = 0; r < NR; ++r) atomicAdd(xs + (int64_t)r * n + gi, -sum[r]);
        }
    }
}

// Column sums of one warp over a 32-column block of a front panel (column c
// at cb + c ld, c < kb): a[r] (lane j) = sum over rows i of W[i, j] v[i + r ld_v],
// the rows taken in passes of SPAN = 32 G rows starting at rows rs, rs + step,
// ... below rend.  Lane l loads row r0 + l of the columns (coalesced per
// column) into registers, writes it transposed into the warp's 32 x 33 tile,
// and lane j accumulates column j over the tile's rows from shared memory: one
// FMA per entry, no shuffle reduction per column.  The columns are read 2^LW
// wide: LW = 5 for a full block, the next pass's loads in flight meanwhile; a
// short block (kb <= 16) is read 16, 8 or 4 wide, one pass then covering
// G = 2^(5-LW) row tiles (tile g in register slots and lanes [g 2^LW,
// (g+1) 2^LW)) whose partial sums of a column are added by shuffles at the
// end -- the FMAs that a 32-wide pass would spend on the missing columns are
// saved.  On return every lane j holds the sums of column j mod 2^LW.
template <class T, int NR, int LW>
__device__ __forceinline__ void warp_col_sums(const T *__restrict__ cb, int64_t ld, int kb, int rs, int rend, int step,
                                              const T *v, int fv, T *tile, int lane, T a[NR]) {
    constexpr int G = 32 >> LW, WM = (1 << LW) - 1;
    constexpr bool PREFETCH = LW == 5;
    T acc[NR], acc2[NR];   // two chains of FMAs per column
#pragma unroll
    for (int r = 0; r < NR; ++r) acc[r] = acc2[r] = T(0);
    T w[32];
    auto load = [&](int r0) {
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            const int i = r0 + 32 * (j >> LW) + lane;
            w[j] = (i < rend && (j & WM) < kb) ? cb[i + (int64_t)(j & WM) * ld] : T(0);
        }
    };
    int r0 = rs;
    if (PREFETCH && r0 < rend) load(r0);
    const int vg = 32 * (lane >> LW);   // this lane's tile within the pass
    for (; r0 < rend; r0 += step) {
        if (!PREFETCH) load(r0);
#pragma unroll
        for (int j = 0; j < 32; ++j) tile[j * 33 + lane] = w[j];
        __syncwarp();
        if (PREFETCH && r0 + step < rend) load(r0 + step);
        const int vb = r0 + vg;
        const T *tl = tile + lane * 33;
        if (r0 + 32 * G <= rend) {
#pragma unroll
            for (int ii = 0; ii < 32; ii += 2) {
                const T t0 = tl[ii], t1 = tl[ii + 1];
#pragma unroll
                for (int r = 0; r < NR; ++r) {
                    acc[r] += t0 * v[vb + ii + r * fv];
                    acc2[r] += t1 * v[vb + ii + 1 + r * fv];
                }
            }
        } else {
            const int cnt = min(32, rend - vb);
            for (int ii = 0; ii < cnt; ++ii) {
                const T t = tl[ii];
#pragma unroll
                for (int r = 0; r < NR; ++r) acc[r] += t * v[vb + ii + r * fv];
            }
        }
        __syncwarp();
    }
#pragma unroll
    for (int r = 0; r < NR; ++r) {
        T x = acc[r] + acc2[r];
#pragma unroll
        for (int o = 1 << LW; o < 32; o <<= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        a[r] = x;
    }
}

template <class T, int NR>
__device__ __forceinline__ void warp_col_sums_short(const T *__restrict__ cb, int64_t ld, int kb, int rs, int rend,
                                                    int passes, const T *v, int fv, T *tile, int lane, T a[NR]) {
    // passes = stride between this warp's passes, counted in passes; a pass spans 32 (32 / 2^LW) rows
    if (kb > 8) warp_col_sums<T, NR, 4>(cb, ld, kb, rs, rend, passes * 64, v, fv, tile, lane, a);
    else if (kb > 4) warp_col_sums<T, NR, 3>(cb, ld, kb, rs, rend, passes * 128, v, fv, tile, lane, a);
    else warp_col_sums<T, NR, 2>(cb, ld, kb, rs, rend, passes * 256, v, fv, tile, lane, a);
}

// Backward substitution for the fronts of one level, one CTA per front.  The
// panel of a front is its pivot rows (the triangle, in partitioned-inverse
// form) over its structure rows (a q x p rectangle).  With u_c = sum over
// structure rows i of W[i, c] x_i, for each block B of 32 pivots from the last
// to the first
//   x_B = L[B,B]^{-T} y_B - W[i,B]^T x_i (later pivot rows i) - u_B.
//   1. u for all columns at once: the rectangle's transposed product has no
//      dependence between blocks, so the warps stream it without a block
//      barrier, warp w taking column blocks w, w + nw, ... (or, when there are
//      fewer blocks than warps, g = nw / blocks warps per block, each every
//      g-th row tile, their partial sums added once).
//   2. the triangle, block by block: the rows of B are negated first so every
//      row enters one column sum with the same sign, the warps take row tiles
//      of the pivot rows from B on, and x_B = -(sum + u_B).
// One FMA per stored entry; no serial triangular solve remains.
template <class T, int NR>
__global__ void __launch_bounds__(SWEEP_MAX_THREADS) k_bwd(const int *__restrict__ fronts, const FrontDesc *__restrict__ D,
                                             const T *__restrict__ L, const int *__restrict__ rows, T *__restrict__ x,
                                             int kcols, int c0) {
    extern __shared__ unsigned char smraw[];
    const FrontDesc d = D[fronts[blockIdx.x]];
    const int p = d.p, f = d.p + d.q, n = d.vlen;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    T *v = reinterpret_cast<T *>(smraw);      // the front's vector, f x NR
    T *u = v + (int64_t)f * NR;                 // structure-row sums per pivot column, p x NR
    T *red = u + (int64_t)p * NR;               // NR x nw x 32 partial column sums
    T *tile = red + 32 * NR * nw + warp * (32 * 33);   // this warp's transposed row tile
    T *xs = x + d.vec_off * kcols + (int64_t)c0 * n;
    for (int i = threadIdx.x; i < f; i += blockDim.x)
#pragma unroll
        for (int r = 0; r < NR; ++r)
            v[i + r * f] = i < p ? xs[(int64_t)r * n + d.first + i] : xs[(int64_t)r * n + rows[d.row_off + i]];
    if (p == 0) return;
    const T *Lp = L + d.l_off;
    const int nbf = p >> 5, kl = p & 31, nb = nbf + (kl ? 1 : 0);
    // 1. structure rows
    if (f > p) {
        const int g = nb >= nw ? 1 : nw / nb, cstep = nw / g, c_first = warp / g, sub = warp % g;
        __syncthreads();
        T a[NR];
        int cb = c_first;
        for (; cb < nbf; cb += cstep) {
            warp_col_sums<T, NR, 5>(Lp + (int64_t)32 * cb * f, f, 32, p + 32 * sub, f, 32 * g, v, f, tile, lane, a);
            if (g == 1) {
#pragma unroll
                for (int r = 0; r < NR; ++r) u[32 * cb + lane + r * p] = a[r];
            } else {
#pragma unroll
                for (int r = 0; r < NR; ++r) red[(r * nw + warp) * 32 + lane] = a[r];
            }
        }
        if (cb == nbf && kl > 0) {
            // the short last block, read narrow when it has at most 16 columns
            if (kl > 16) {
                warp_col_sums<T, NR, 5>(Lp + (int64_t)32 * cb * f, f, kl, p + 32 * sub, f, 32 * g, v, f, tile, lane,
                                        a);
            } else {
                const int span = 32 * (32 >> (kl > 8 ? 4 : (kl > 4 ? 3 : 2)));
                warp_col_sums_short<T, NR>(Lp + (int64_t)32 * cb * f, f, kl, p + span * sub, f, g, v, f, tile, lane,
                                           a);
            }
            if (g == 1) {
                if (lane < kl)
#pragma unroll
                    for (int r = 0; r < NR; ++r) u[32 * cb + lane + r * p] = a[r];
            } else {
#pragma unroll
                for (int r = 0; r < NR; ++r) red[(r * nw + warp) * 32 + lane] = a[r];
            }
        }
        __syncthreads();
        if (g > 1)
            for (int c = threadIdx.x; c < 32 * NR * nb; c += blockDim.x) {
                const int r = c / (32 * nb), cc = c % (32 * nb), j = cc & 31, b = cc >> 5;
                if (cc >= p) continue;
                T s = T(0);
                for (int k = 0; k < g; ++k) s += red[(r * nw + b * g + k) * 32 + j];
                u[cc + r * p] = s;
            }
    } else {
        for (int c = threadIdx.x; c < p * NR; c += blockDim.x) u[c] = T(0);
    }
    __syncthreads();
    // 2. the triangle
    int jb = ((p - 1) / 32) * 32;
    if (threadIdx.x < 32 * NR) {
        const int j = threadIdx.x & 31, r = threadIdx.x >> 5;
        if (j < p - jb) v[jb + j + r * f] = -v[jb + j + r * f];
    }
    __syncthreads();
    // column sums of the block at jb (partial per warp in red) -> x_B; negate the next block's rows
    auto finish = [&](int jb, int kb) {
        __syncthreads();
        if (threadIdx.x < 32 * NR) {
            const int j = threadIdx.x & 31, r = threadIdx.x >> 5;
            T s = T(0);
            for (int ww = 0; ww < nw; ++ww) s += red[(r * nw + ww) * 32 + j];
            if (j < kb) v[jb + j + r * f] = -(s + u[jb + j + r * p]);
            // the next block's rows (read from the next step on) enter its sum negated
            if (jb >= 32) v[jb - 32 + j + r * f] = -v[jb - 32 + j + r * f];
        }
        __syncthreads();
    };
    T a[NR];
    if (kl > 0 && kl <= 16) {
        // a short last block, read narrow (once per front, before the full blocks)
        const int span = 32 * (32 >> (kl > 8 ? 4 : (kl > 4 ? 3 : 2)));
        warp_col_sums_short<T, NR>(Lp + (int64_t)jb * f, f, kl, jb + span * warp, p, nw, v, f, tile, lane, a);
#pragma unroll
        for (int r = 0; r < NR; ++r) red[(r * nw + warp) * 32 + lane] = a[r];
        finish(jb, kl);
        jb -= 32;
    }
    for (; jb >= 0; jb -= 32) {
        const int kb = min(32, p - jb);
        warp_col_sums<T, NR, 5>(Lp + (int64_t)jb * f, f, kb, jb + 32 * warp, p, 32 * nw, v, f, tile, lane, a);
#pragma unroll
        for (int r = 0; r < NR; ++r) red[(r * nw + warp) * 32 + lane] = a[r];
        finish(jb, kb);
    }
    for (int i = threadIdx.x; i < p; i += blockDim.x)
#pragma unroll
        for (int r = 0; r < NR; ++r) xs[(int64_t)r * n + d.first + i] = v[i + r * f];
}

// Backward substitution with per-column shuffle reductions, used for the FP32
// factors: for each block B of 32 pivots from the last to the first, one
// reduction down each column of the block over the rows from B to the end of
// the front (the rows of B with +, the rows below with -); warp w owns the
// columns w, w + 8, ..., its lanes stride the rows with 8 loads in flight, and
// a shuffle tree adds the lanes.  Its adds cost little where the sweep is
// bound by HBM (FP32), and its 32 registers and small shared memory keep many
// CTAs and loads in flight; the FP64 sweep, bound by the FP64 pipe, uses k_bwd.
template <class T, int NR>
__global__ void __launch_bounds__(SWEEP_MAX_THREADS) k_bwd_shfl(const int *__restrict__ fronts, const FrontDesc *__restrict__ D,
                                             const T *__restrict__ L, const int *__restrict__ rows, T *__restrict__ x,
                                             int kcols, int c0) {
    extern __shared__ unsigned char smraw[];
    const FrontDesc d = D[fronts[blockIdx.x]];
    const int p = d.p, f = d.p + d.q, n = d.vlen;
    T *v = reinterpret_cast<T *>(smraw);
    T *red = v + (int64_t)f * NR;   // 32 x NR column results of the block
    T *xs = x + d.vec_off * kcols + (int64_t)c0 * n;
    for (int i = threadIdx.x; i < f; i += blockDim.x)
#pragma unroll
        for (int r = 0; r < NR; ++r)
            v[i + r * f] = i < p ? xs[(int64_t)r * n + d.first + i] : xs[(int64_t)r * n + rows[d.row_off + i]];
    __syncthreads();
    if (p == 0) return;
    const T *Lp = L + d.l_off;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int jb = ((p - 1) / 32) * 32; jb >= 0; jb -= 32) {
        const int kb = min(32, p - jb);
        for (int j = warp; j < kb; j += nw) {
            const T *col = Lp + (int64_t)(jb + j) * f;
            T acc[NR];
            {
                // rows of B: L[B,B]^{-1}[i, j] y_i for i >= j, negated here and restored below
                const bool in = lane >= j && lane < kb;
                const T l = in ? col[jb + lane] : T(0);
#pragma unroll
                for (int r = 0; r < NR; ++r) acc[r] = -(l * v[jb + (in ? lane : 0) + r * f]);
            }
            int i = jb + kb + lane;
            // rows below B: + W[i, j] x_i, 8 independent loads per lane in flight
            for (; i + 7 * 32 < f; i += 8 * 32) {
                T l[8];
#pragma unroll
                for (int t = 0; t < 8; ++t) l[t] = col[i + 32 * t];
#pragma unroll
                for (int t = 0; t < 8; ++t)
#pragma unroll
                    for (int r = 0; r < NR; ++r) acc[r] += l[t] * v[i + 32 * t + r * f];
            }
            for (; i < f; i += 32) {
                const T l = col[i];
#pragma unroll
                for (int r = 0; r < NR; ++r) acc[r] += l * v[i + r * f];
            }
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                T a = acc[r];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
                if (lane == 0) red[j + 32 * r] = -a;
            }
        }
        __syncthreads();
        if (threadIdx.x < 32 * NR) {
            const int j = threadIdx.x & 31, r = threadIdx.x >> 5;
            if (j < kb) v[jb + j + r * f] = red[j + 32 * r];
        }
        __syncthreads();
    }
    for (int i = threadIdx.x; i < p; i += blockDim.x)
#pragma unroll
        for (int r = 0; r < NR; ++r) xs[(int64_t)r * n + d.first + i] = v[i + r * f];
}

// Shared memory of the sweeps.  Forward: the front vector (f x NR) and the
// copy of x_B (32 x NR), plus the static inverse block.  Backward: the front
// vector, the partial column sums (NR x nw x 32) and one 32 x 33 tile per warp,
// so its block size shrinks on levels whose largest front would not fit.  The
// dynamic limit of every variant is raised once per device to all that a CTA
// may hold; build_plan calls sweep_smem_for_plan for every variant, so no
// attribute is ever changed while a stream is being captured.
constexpr size_t SMEM_PER_CTA = 227 * 1024;

template <class T, int NR>
static size_t sweep_static_smem() {
    static const size_t v = [] {
        cudaFuncAttributes a{}, b{};
        GL_CUDA(cudaFuncGetAttributes(&a, k_fwd<T, NR, fwd_split<T>()>));
        GL_CUDA(cudaFuncGetAttributes(&b, k_bwd<T, NR>));
        return std::max<size_t>(1, std::max(a.sharedSizeBytes, b.sharedSizeBytes));
    }();
    return v;
}

template <class T, int NR>
static size_t fwd_dyn_smem(int f) {
    // front vector and the blocks' x_B (p <= f)
    return (2 * (size_t)std::max(f, 1)) * NR * sizeof(T);
}

template <class T, int NR>
static size_t bwd_dyn_smem(int f, int nthreads) {
    // front vector and structure-row sums (p <= f), partial sums, one tile per warp
    const size_t nw = (size_t)nthreads / 32;
    return ((size_t)std::max(f, 1) * NR * 2 + 32 * NR * nw + 33 * 32 * nw) * sizeof(T);
}

template <class T, int NR>
constexpr int bwd_min_threads() {
    return 32 * NR;   // the column sums of the block are finished by 32 NR threads
}

template <class T, int NR>
static bool sweep_fits(int max_f) {
    const size_t lim = SMEM_PER_CTA - sweep_static_smem<T, NR>();
    return fwd_dyn_smem<T, NR>(max_f) <= lim && bwd_dyn_smem<T, NR>(max_f, bwd_min_threads<T, NR>()) <= lim;
}

// Threads per CTA of the backward sweep on a level: the wanted count, halved
// while the level's largest front does not fit.
template <class T, int NR>
static int bwd_threads(int max_f, int want) {
    const size_t lim = SMEM_PER_CTA - sweep_static_smem<T, NR>();
    int nt = want;
    while (nt > bwd_min_threads<T, NR>() && bwd_dyn_smem<T, NR>(max_f, nt) > lim) nt /= 2;
    return nt;
}

template <class T, int NR>
static void ensure_sweep_smem(int max_f) {
    static SmemLimit limit;
    if (!sweep_fits<T, NR>(max_f)) return;
    raise_smem_limit(limit, SMEM_PER_CTA - sweep_static_smem<T, NR>(), [](size_t v) {
        GL_CUDA(cudaFuncSetAttribute(k_fwd<T, NR, fwd_split<T>()>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)v));
        GL_CUDA(cudaFuncSetAttribute(k_bwd<T, NR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)v));
        GL_CUDA(cudaFuncSetAttribute(k_bwd_shfl<T, NR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)v));
    });
}

template <class T, int NR>
static size_t bwd_shfl_dyn_smem(int f) {
    return ((size_t)std::max(f, 1) + 32) * NR * sizeof(T);
}

void sweep_smem_for_plan(int max_f) {
    ensure_sweep_smem<double, 1>(max_f);
    ensure_sweep_smem<double, 2>(max_f);
    ensure_sweep_smem<double, 4>(max_f);
    ensure_sweep_smem<float, 1>(max_f);
    ensure_sweep_smem<float, 2>(max_f);
    ensure_sweep_smem<float, 4>(max_f);
}

void level_clock_enable(FactorPlan &P, bool on) {
    LevelClock &K = P.clock;
    const size_t nlev = P.levels.size();
    if (on && K.ev.size() != 2 * nlev + 1) {
        for (cudaEvent_t e : K.ev)
            if (e) cudaEventDestroy(e);
        K.ev.assign(2 * nlev + 1, nullptr);
        for (cudaEvent_t &e : K.ev) GL_CUDA(cudaEventCreate(&e));
    }
    K.fwd_ms.assign(nlev, 0.0);
    K.bwd_ms.assign(nlev, 0.0);
    K.calls = 0;
    K.on = on;
}

// Events e[0..2 nlev]: e[nlev-1-d] before the forward launch of depth d,
// e[nlev+d] before its backward launch, e[2 nlev] after the last launch.
static void level_clock_fold(const FactorPlan &P) {
    LevelClock &K = P.clock;
    const int nlev = (int)P.levels.size();
    GL_CUDA(cudaEventSynchronize(K.ev[2 * nlev]));
    for (int d = 0; d < nlev; ++d) {
        float a = 0, b = 0;
        GL_CUDA(cudaEventElapsedTime(&a, K.ev[nlev - 1 - d], K.ev[nlev - d]));
        GL_CUDA(cudaEventElapsedTime(&b, K.ev[nlev + d], K.ev[nlev + d + 1]));
        K.fwd_ms[d] += a;
        K.bwd_ms[d] += b;
    }
    K.calls += 1;
}

static int sweep_threads(const Level &Lv, bool bwd) {
    if (Lv.fronts.size() < (size_t)SWEEP_WIDE_BELOW) return bwd ? GL_SWEEP_BWD_WIDE_THREADS : GL_SWEEP_FWD_WIDE_THREADS;
    if (Lv.max_f <= GL_SWEEP_SMALL_F) return bwd ? GL_SWEEP_BWD_SMALL_THREADS : GL_SWEEP_FWD_SMALL_THREADS;
    return bwd ? GL_SWEEP_BWD_THREADS : GL_SWEEP_FWD_THREADS;
}

// One level's forward or backward sweep over the fronts fr[0..nf) of that level.
template <class T, int NR>
static void launch_fwd(const FactorPlan &P, const Level &Lv, const int *fr, unsigned nf, const T *L, T *x, int kcols,
                       int c0, cudaStream_t s) {
    if (nf == 0) return;
    const size_t sm = fwd_dyn_smem<T, NR>(Lv.max_f);
    k_fwd<T, NR, fwd_split<T>()><<<nf, sweep_threads(Lv, false), sm, s>>>(fr, P.d_fr.p, L, P.d_rows.p, x, kcols,
                                                                         c0);
}

template <class T, int NR>
static void launch_bwd(const FactorPlan &P, const Level &Lv, const int *fr, unsigned nf, const T *L, T *x, int kcols,
                       int c0, cudaStream_t s) {
    if (nf == 0) return;
    const int want = sweep_threads(Lv, true);
    if (sizeof(T) == 4) {
        const size_t sm = bwd_shfl_dyn_smem<T, NR>(Lv.max_f);
        k_bwd_shfl<T, NR><<<nf, want, sm, s>>>(fr, P.d_fr.p, L, P.d_rows.p, x, kcols, c0);
    } else {
        const int nt = bwd_threads<T, NR>(Lv.max_f, want);
        const size_t sm = bwd_dyn_smem<T, NR>(Lv.max_f, nt);
        k_bwd<T, NR><<<nf, nt, sm, s>>>(fr, P.d_fr.p, L, P.d_rows.p, x, kcols, c0);
    }
}

static HalfStreams &half_streams(const FactorPlan &P) {
    if (!P.hs) {
        auto h = std::make_unique<HalfStreams>();
        int lo = 0, hi = 0;
        GL_CUDA(cudaDeviceGetStreamPriorityRange(&lo, &hi));
        for (int k = 0; k < 2; ++k) {
            GL_CUDA(cudaStreamCreateWithPriority(&h->hi[k], cudaStreamNonBlocking, hi));
            GL_CUDA(cudaStreamCreateWithPriority(&h->lo[k], cudaStreamNonBlocking, lo));
        }
        GL_CUDA(cudaEventCreateWithFlags(&h->fork, cudaEventDisableTiming));
        for (cudaEvent_t &e : h->ev) GL_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        P.hs = std::move(h);
    }
    return *P.hs;
}

// Overlapped sweeps of the two halves of the subdomains (FactorPlan::overlap_top
// = k > 0).  Half h: deep forward levels (depth >= k) on lo[h], then its top
// levels (forward to the root and backward down to depth k - 1) on hi[h],
// then its deep backward levels on lo[h].  The second half's deep forward
// levels start when the first half enters its top levels.  The halves hold
// disjoint subdomains, so they share no data.
template <class T, int NR>
static void solve_levels_overlap(const FactorPlan &P, const T *L, T *x, int kcols, int c0, cudaStream_t s) {
    HalfStreams &H = half_streams(P);
    const int nlev = (int)P.levels.size(), k = std::min(P.overlap_top, nlev);
    GL_CUDA(cudaEventRecord(H.fork, s));
    for (int h = 0; h < 2; ++h) {
        GL_CUDA(cudaStreamWaitEvent(H.lo[h], H.fork, 0));
        GL_CUDA(cudaStreamWaitEvent(H.hi[h], H.fork, 0));
    }
    auto part = [&](int h, int d, const int *&fr, unsigned &nf) {
        const Level &Lv = P.levels[d];
        const unsigned na = (unsigned)P.half_fronts[d];
        fr = Lv.d_fronts.p + (h == 0 ? 0 : na);
        nf = h == 0 ? na : (unsigned)Lv.fronts.size() - na;
    };
    // ev[3h]: half h reached its top levels; ev[3h+1]: its top levels are done; ev[3h+2]: all done
    for (int h = 0; h < 2; ++h) {
        if (h == 1) GL_CUDA(cudaStreamWaitEvent(H.lo[1], H.ev[0], 0));
        for (int d = nlev - 1; d >= k; --d) {
            const int *fr; unsigned nf;
            part(h, d, fr, nf);
            launch_fwd<T, NR>(P, P.levels[d], fr, nf, L, x, kcols, c0, H.lo[h]);
        }
        GL_CUDA(cudaEventRecord(H.ev[3 * h], H.lo[h]));
        GL_CUDA(cudaStreamWaitEvent(H.hi[h], H.ev[3 * h], 0));
        for (int d = k - 1; d >= 0; --d) {
            const int *fr; unsigned nf;
            part(h, d, fr, nf);
            launch_fwd<T, NR>(P, P.levels[d], fr, nf, L, x, kcols, c0, H.hi[h]);
        }
        for (int d = 0; d < k; ++d) {
            const int *fr; unsigned nf;
            part(h, d, fr, nf);
            launch_bwd<T, NR>(P, P.levels[d], fr, nf, L, x, kcols, c0, H.hi[h]);
        }
        GL_CUDA(cudaEventRecord(H.ev[3 * h + 1], H.hi[h]));
    }
    for (int h = 0; h < 2; ++h) {
        GL_CUDA(cudaStreamWaitEvent(H.lo[h], H.ev[3 * h + 1], 0));
        for (int d = k; d < nlev; ++d) {
            const int *fr; unsigned nf;
            part(h, d, fr, nf);
            launch_bwd<T, NR>(P, P.levels[d], fr, nf, L, x, kcols, c0, H.lo[h]);
        }
        GL_CUDA(cudaEventRecord(H.ev[3 * h + 2], H.lo[h]));
        GL_CUDA(cudaStreamWaitEvent(s, H.ev[3 * h + 2], 0));
    }
    GL_CUDA(cudaGetLastError());
}

template <class T, int NR>
static void solve_levels(const FactorPlan &P, const T *L, T *x, int kcols, int c0, cudaStream_t s) {
    ensure_sweep_smem<T, NR>(P.max_f);
    const int nlev = (int)P.levels.size();
    const bool timed = NR == 1 && kcols == 1 && P.clock.on && P.clock.ev.size() == 2 * (size_t)nlev + 1;
    if (NR == 1 && kcols == 1 && P.overlap_top > 0 && !timed && P.n_sub >= 2) {
        solve_levels_overlap<T, NR>(P, L, x, kcols, c0, s);
        return;
    }
    auto mark = [&](int k) {
        if (timed) GL_CUDA(cudaEventRecord(P.clock.ev[k], s));
    };
    for (int dpt = nlev - 1; dpt >= 0; --dpt) {
        mark(nlev - 1 - dpt);
        const Level &Lv = P.levels[dpt];
        launch_fwd<T, NR>(P, Lv, Lv.d_fronts.p, (unsigned)Lv.fronts.size(), L, x, kcols, c0, s);
    }
    for (int dpt = 0; dpt < nlev; ++dpt) {
        mark(nlev + dpt);
        const Level &Lv = P.levels[dpt];
        launch_bwd<T, NR>(P, Lv, Lv.d_fronts.p, (unsigned)Lv.fronts.size(), L, x, kcols, c0, s);
    }
    GL_CUDA(cudaGetLastError());
    if (timed) {
        mark(2 * nlev);
        level_clock_fold(P);
    }
}

template <class T>
void factor_solve(const FactorPlan &P, const T *L, T *x, int kcols, cudaStream_t s) {
    const int nr = sweep_fits<T, 4>(P.max_f) ? 4 : (sweep_fits<T, 2>(P.max_f) ? 2 : 1);
    if (!sweep_fits<T, 1>(P.max_f)) fail(GL_ERR_INVALID_ARG, "factor_solve: front too large for shared memory");
    int c0 = 0;
    while (c0 < kcols) {
        int left = kcols - c0;
        if (nr >= 4 && left >= 4) { solve_levels<T, 4>(P, L, x, kcols, c0, s); c0 += 4; }
        else if (nr >= 2 && left >= 2) { solve_levels<T, 2>(P, L, x, kcols, c0, s); c0 += 2; }
        else { solve_levels<T, 1>(P, L, x, kcols, c0, s); c0 += 1; }
    }
}

template void factor_solve<double>(const FactorPlan &, const double *, double *, int, cudaStream_t);
template void factor_solve<float>(const FactorPlan &, const float *, float *, int, cudaStream_t);

// ----------------------------------------------------------------- local <-> global

template <class T>
__global__ void k_gather(int64_t n, const int64_t *__restrict__ gdof, const double *__restrict__ r, T *__restrict__ xl) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) xl[i] = (T)r[gdof[i]];
}

template <class T>
__global__ void k_scatter_add(int64_t n, const int64_t *__restrict__ gdof, const T *__restrict__ xl, double *__restrict__ z) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) atomicAdd(z + gdof[i], (double)xl[i]);
}

template <class T>
void gather_local(const FactorPlan &P, const double *r, T *xl, cudaStream_t s) {
    if (!P.n_local) return;
    k_gather<T><<<(unsigned)((P.n_local + 255) / 256), 256, 0, s>>>(P.n_local, P.d_gdof.p, r, xl);
    GL_CUDA(cudaGetLastError());
}
template <class T>
void scatter_add_local(const FactorPlan &P, const T *xl, double *z, cudaStream_t s) {
    if (!P.n_local) return;
    k_scatter_add<T><<<(unsigned)((P.n_local + 255) / 256), 256, 0, s>>>(P.n_local, P.d_gdof.p, xl, z);
    GL_CUDA(cudaGetLastError());
}
template void gather_local<double>(const FactorPlan &, const double *, double *, cudaStream_t);
template void gather_local<float>(const FactorPlan &, const double *, float *, cudaStream_t);
template void scatter_add_local<double>(const FactorPlan &, const double *, double *, cudaStream_t);
template void scatter_add_local<float>(const FactorPlan &, const float *, double *, cudaStream_t);

// ----------------------------------------------------------------- dense (coarse) inverse

// K^{-1} of a dense SPD matrix through the same partial Cholesky: factoring the
// p = n pivots of the 2n x 2n front [[A_s, I], [I, 0]] leaves the Schur
// complement 0 - I A_s^{-1} I = -A_s^{-1} in the trailing block, where
// A_s = D A D is A scaled to unit diagonal (D = diag(A)^{-1/2}); then
// A^{-1} = D A_s^{-1} D.  With drop > 0 a pivot of |v| <= drop (on the unit
// diagonal scale) marks its column as linearly dependent on the earlier ones:
// the column is left out of the factor, its row and column of the result are
// zero, and the result is the inverse of A on the kept columns -- a
// generalised inverse of A when the dropped columns lie in the span of the
// kept ones (a zero column of A has a zero scaled pivot and is dropped too).
__device__ __forceinline__ double unit_diag_scale(const double *A, int n, int64_t i) {
    const double d = A[i + i * (int64_t)n];
    return d > 0.0 ? 1.0 / sqrt(d) : 0.0;
}

__global__ void k_aug_init(const double *__restrict__ A, int n, double *__restrict__ F) {
    const int64_t m = 2 * (int64_t)n;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < m * m; idx += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = idx % m, j = idx / m;
        double v = 0.0;
        if (i < n && j < n) {
            const double di = unit_diag_scale(A, n, i), dj = unit_diag_scale(A, n, j);
            v = (di == 0.0 || dj == 0.0) ? 0.0 : A[i + j * n] * di * dj;
        } else if (j < n && i - n == j) {
            v = 1.0;
        }
        F[idx] = v;
    }
}

__global__ void k_extract_inv(const double *__restrict__ A, const double *__restrict__ F, int n,
                              double *__restrict__ Ainv) {
    const int64_t m = 2 * (int64_t)n;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < (int64_t)n * n;
         idx += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = idx % n, j = idx / n;
        int64_t a = i > j ? i : j, b = i > j ? j : i;   // lower triangle of the trailing block
        Ainv[idx] = -F[(n + a) + (n + b) * m] * unit_diag_scale(A, n, i) * unit_diag_scale(A, n, j);
    }
}

int dense_inverse(const double *A, int n, double *Ainv, int *d_err, cudaStream_t s, double drop) {
    DBuf<FrontDesc> d;
    DBuf<int> idx, drops;
    FrontDesc f{};
    f.p = n;
    f.q = n;
    f.vlen = 2 * n;
    f.parent = -1;
    d.upload(std::vector<FrontDesc>{f}, s);
    idx.upload(std::vector<int>{0}, s);
    drops.alloc(1);
    drops.zero(s);
    DBuf<double> F;
    F.alloc((size_t)4 * n * n);
    k_aug_init<<<1024, 256, 0, s>>>(A, n, F.p);
    GL_CUDA(cudaGetLastError());
    partial_cholesky_level(idx.p, 1, d.p, n, 2 * n, F.p, false, d_err, s, drop, drops.p);
    k_extract_inv<<<1024, 256, 0, s>>>(A, F.p, n, Ainv);
    GL_CUDA(cudaGetLastError());
    int h = 0;
    GL_CUDA(cudaMemcpyAsync(&h, drops.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    GL_CUDA(cudaStreamSynchronize(s));
    return h;
}

// Block-diagonal version: for each block b, y[o_b : o_b + n_b] = A_b x[o_b : o_b + n_b],
// A_b stored column-major at aoff[b]; one warp per output row.
__global__ void k_symv_blocks(const double *__restrict__ A, const int64_t *__restrict__ aoff,
                              const int *__restrict__ voff, const int *__restrict__ nb, int nblk,
                              const double *__restrict__ x, double *__restrict__ y, int total) {
    const int lane = threadIdx.x & 31;
    const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (row >= total) return;
    int lo = 0, hi = nblk - 1;   // block containing this row
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (voff[mid] <= row) lo = mid;
        else hi = mid - 1;
    }
    const int b = lo, n = nb[b], i = row - voff[b];
    const double *col = A + aoff[b] + (int64_t)i * n;
    const double *xb = x + voff[b];
    double acc = 0.0;
    for (int j = lane; j < n; j += 32) acc += col[j] * xb[j];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) y[row] = acc;
}

void dense_symv_blocks(const double *A, const int64_t *aoff, const int *voff, const int *nb, int nblk, int total,
                       const double *x, double *y, cudaStream_t s) {
    if (total <= 0) return;
    k_symv_blocks<<<(total + 7) / 8, 256, 0, s>>>(A, aoff, voff, nb, nblk, x, y, total);
    GL_CUDA(cudaGetLastError());
}

}  // namespace gl
