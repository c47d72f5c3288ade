// Host symbolic phase of the local subdomain factorisations (Section 2.3: the
// subdomain problems with zero displacement on the artificial boundary are
// solved by a direct method).
//
// Geometric nested dissection on the structured Q2 node grid of one
// subdomain: a region (a box of active nodes) is split by a plane of nodes at
// an even (element-vertex) index strictly inside it -- no element spans such a
// plane, so it separates the two halves -- until the region holds at most
// `leaf_nodes` nodes.  Each separator and each leaf becomes one supernode;
// children precede parents (postorder), which is also the elimination order.
// The structure of a supernode is the set of active nodes adjacent to its
// subtree region, i.e. the enclosing box of all elements touching the region
// minus the region itself (all of them lie on ancestor separators).  The
// front of a supernode = its pivots followed by its structure rows.
//
// Periodic width (the last width plane identified with the first; the
// subdomain then spans the width): the first plane is the root separator, a
// supernode with one child, the rest of the box below it dissected as usual.
// Wherever a node of the last plane appears -- in a region's neighbourhood or
// among an element's nodes -- its partner on the first plane stands for it,
// and the root also assembles the elements of the last width layer.
#include <algorithm>
#include <cstdio>

#include "gl_internal.h"

namespace gl {

namespace {

struct Box {
    int lo[3], hi[3];   // inclusive node index ranges
    int64_t count() const {
        int64_t c = 1;
        for (int d = 0; d < 3; ++d) c *= (hi[d] >= lo[d]) ? (hi[d] - lo[d] + 1) : 0;
        return c;
    }
};

struct Builder {
    const MeshHost &m;
    const std::vector<uint8_t> &is_dir;
    Box active;
    int leaf_nodes;
    SubSymbolic &S;
    std::vector<int> node_first;   // per node of the active box: first local DOF index, -1 if none
    std::vector<uint8_t> node_ndof;
    std::vector<uint8_t> node_comp_mask;
    std::vector<Box> region;       // subtree region per supernode
    std::vector<Box> piv_box;      // pivot node box per supernode
    int next_local = 0;

    Builder(const MeshHost &m_, const std::vector<uint8_t> &d, const Box &a, int leaf, SubSymbolic &s)
        : m(m_), is_dir(d), active(a), leaf_nodes(leaf), S(s) {
        node_first.assign(active.count(), -1);
        node_ndof.assign(active.count(), 0);
        node_comp_mask.assign(active.count(), 0);
    }

    int64_t lidx(int x, int y, int z) const {
        return (int64_t)(x - active.lo[0]) +
               (int64_t)(active.hi[0] - active.lo[0] + 1) *
                   ((int64_t)(y - active.lo[1]) + (int64_t)(active.hi[1] - active.lo[1] + 1) * (z - active.lo[2]));
    }
    int64_t gnode(int x, int y, int z) const { return (int64_t)x + (int64_t)m.NX * ((int64_t)y + (int64_t)m.NY * z); }
    // the node that carries the DOFs of (x, y, z): its first-plane partner on the last width plane
    int wrap_y(int y) const { return (m.periodic && y == m.NY - 1) ? 0 : y; }

    // numbers the active DOFs of the nodes of box b (x fastest), returns count
    int number_box(const Box &b) {
        int start = next_local;
        for (int z = b.lo[2]; z <= b.hi[2]; ++z)
            for (int y = b.lo[1]; y <= b.hi[1]; ++y)
                for (int x = b.lo[0]; x <= b.hi[0]; ++x) {
                    int64_t g = gnode(x, y, z);
                    int64_t li = lidx(x, y, z);
                    uint8_t mask = 0, nd = 0;
                    for (int c = 0; c < 3; ++c)
                        if (!is_dir[3 * g + c]) {
                            mask |= (uint8_t)(1u << c);
                            ++nd;
                        }
                    node_comp_mask[li] = mask;
                    node_ndof[li] = nd;
                    if (nd) {
                        node_first[li] = next_local;
                        for (int c = 0; c < 3; ++c)
                            if (mask & (1u << c)) S.gdof.push_back(3 * g + c);
                        next_local += nd;
                    }
                }
        return next_local - start;
    }

    int new_supernode(const Box &reg, const Box &piv, int depth, int c0, int c1) {
        Supernode s{};
        s.first = next_local;
        s.p = number_box(piv);
        s.depth = depth;
        s.parent = -1;
        s.child[0] = c0;
        s.child[1] = c1;
        for (int d = 0; d < 3; ++d) {
            s.box[2 * d] = reg.lo[d];
            s.box[2 * d + 1] = reg.hi[d];
        }
        int id = (int)S.sn.size();
        S.sn.push_back(s);
        region.push_back(reg);
        piv_box.push_back(piv);
        if (c0 >= 0) S.sn[c0].parent = id;
        if (c1 >= 0) S.sn[c1].parent = id;
        S.max_depth = std::max(S.max_depth, depth);
        return id;
    }

    int nd(const Box &R, int depth) {
        // pick the longest axis that has an even index strictly inside
        int best = -1, best_len = 0;
        for (int d = 0; d < 3; ++d) {
            int len = R.hi[d] - R.lo[d] + 1;
            int first_even = (R.lo[d] + 1) + ((R.lo[d] + 1) & 1);
            if (first_even >= R.hi[d]) continue;
            if (len > best_len) {
                best_len = len;
                best = d;
            }
        }
        if (R.count() <= leaf_nodes || best < 0) return new_supernode(R, R, depth, -1, -1);
        int mid = (R.lo[best] + R.hi[best]) / 2;
        int s = mid & ~1;
        if (s <= R.lo[best]) s += 2;
        if (s >= R.hi[best]) s -= 2;
        Box L = R, Rr = R, P = R;
        L.hi[best] = s - 1;
        Rr.lo[best] = s + 1;
        P.lo[best] = P.hi[best] = s;
        int c0 = nd(L, depth + 1);
        int c1 = nd(Rr, depth + 1);
        return new_supernode(R, P, depth, c0, c1);
    }

    Box expand(const Box &R) const {
        Box E = R;
        for (int d = 0; d < 3; ++d) {
            E.lo[d] = R.lo[d] - ((R.lo[d] & 1) ? 1 : 2);
            E.hi[d] = R.hi[d] + ((R.hi[d] & 1) ? 1 : 2);
            E.lo[d] = std::max(E.lo[d], active.lo[d]);
            E.hi[d] = std::min(E.hi[d], active.hi[d]);
        }
        return E;
    }

    static bool inside(const Box &b, int x, int y, int z) {
        return x >= b.lo[0] && x <= b.hi[0] && y >= b.lo[1] && y <= b.hi[1] && z >= b.lo[2] && z <= b.hi[2];
    }
};

}  // namespace

void build_symbolic(const MeshHost &m, const SubBox &b, const std::vector<uint8_t> &dof_is_dir, bool neumann,
                    int leaf_nodes, SubSymbolic &S) {
    S = SubSymbolic();
    Box A;
    for (int d = 0; d < 3; ++d) {
        A.lo[d] = b.nbox[2 * d];
        A.hi[d] = b.nbox[2 * d + 1];
        if (!neumann) {
            if (b.art[2 * d]) A.lo[d] += 1;
            if (b.art[2 * d + 1]) A.hi[d] -= 1;
        }
    }
    if (A.count() <= 0) fail(GL_ERR_INVALID_ARG, "empty subdomain");
    Builder B(m, dof_is_dir, A, leaf_nodes, S);
    const bool wrap = m.periodic;
    if (wrap) {
        if (A.lo[1] != 0 || A.hi[1] != m.NY - 1) fail(GL_ERR_INVALID_ARG, "periodic width: a subdomain must span the width");
        Box P = A, Rr = A;
        P.hi[1] = 0;
        Rr.lo[1] = 1;
        const int c0 = B.nd(Rr, 1);
        const int root = B.new_supernode(A, P, 0, c0, -1);
        (void)root;
    } else {
        B.nd(A, 0);
    }
    S.n = B.next_local;

    // structure rows
    const int nsn = (int)S.sn.size();
    std::vector<std::vector<int>> structs(nsn);
    for (int i = 0; i < nsn; ++i) {
        const Box &R = B.region[i];
        Box E = B.expand(R);
        std::vector<int> &rows = structs[i];
        for (int z = E.lo[2]; z <= E.hi[2]; ++z)
            for (int y = E.lo[1]; y <= E.hi[1]; ++y)
                for (int x = E.lo[0]; x <= E.hi[0]; ++x) {
                    const int yw = B.wrap_y(y);
                    if (Builder::inside(R, x, yw, z)) continue;
                    int64_t li = B.lidx(x, yw, z);
                    int f = B.node_first[li];
                    for (int k = 0; k < B.node_ndof[li]; ++k) rows.push_back(f + k);
                }
        std::sort(rows.begin(), rows.end());
        rows.erase(std::unique(rows.begin(), rows.end()), rows.end());
        Supernode &s = S.sn[i];
        if (!rows.empty() && rows.front() < s.first + s.p)
            fail(GL_ERR_STATE, "symbolic: structure row precedes its supernode");
        s.q = (int)rows.size();
    }
    // offsets, rows, relative maps
    int64_t loff = 0, roff = 0;
    for (int i = 0; i < nsn; ++i) {
        Supernode &s = S.sn[i];
        int f = s.p + s.q;
        s.l_off = loff;
        loff += (int64_t)f * s.p;
        s.row_off = roff;
        roff += f;
        for (int k = 0; k < s.p; ++k) S.rows.push_back(s.first + k);
        S.rows.insert(S.rows.end(), structs[i].begin(), structs[i].end());
    }
    S.l_size = loff;
    for (int i = 0; i < nsn; ++i) {
        Supernode &s = S.sn[i];
        s.rel_off = (int64_t)S.rel.size();
        if (s.parent < 0) {
            if (s.q) fail(GL_ERR_STATE, "symbolic: root supernode has structure rows");
            continue;
        }
        const Supernode &P = S.sn[s.parent];
        const std::vector<int> &ps = structs[s.parent];
        for (int g : structs[i]) {
            int pos;
            if (g >= P.first && g < P.first + P.p) {
                pos = g - P.first;
            } else {
                auto it = std::lower_bound(ps.begin(), ps.end(), g);
                if (it == ps.end() || *it != g) fail(GL_ERR_STATE, "symbolic: child row missing from parent front");
                pos = P.p + (int)(it - ps.begin());
            }
            S.rel.push_back(pos);
        }
    }
    // (front, element) assembly pairs
    const int ex0 = b.ebox[0], ex1 = b.ebox[1], ey0 = b.ebox[2], ey1 = b.ebox[3], ez0 = b.ebox[4], ez1 = b.ebox[5];
    for (int i = 0; i < nsn; ++i) {
        Supernode &s = S.sn[i];
        s.emap_off = (int64_t)S.pair_elem.size();
        s.n_elem_pairs = 0;
        if (s.p == 0) continue;
        const Box &P = B.piv_box[i];
        int elo[3], ehi[3];
        const int eb_lo[3] = {ex0, ey0, ez0}, eb_hi[3] = {ex1, ey1, ez1};
        for (int d = 0; d < 3; ++d) {
            // elements e with 2e + 2 >= lo and 2e <= hi, inside the subdomain
            elo[d] = std::max(P.lo[d] <= 2 ? 0 : (P.lo[d] - 1) / 2, eb_lo[d]);
            ehi[d] = std::min(P.hi[d] / 2, eb_hi[d] - 1);
        }
        const std::vector<int> &st = structs[i];
        // element rows of the width to visit: those touching the pivots, and under periodic width
        // the last row for a pivot box on the first plane (its last-plane nodes stand for them)
        std::vector<int> eys;
        for (int ey = elo[1]; ey <= ehi[1]; ++ey) eys.push_back(ey);
        if (wrap && P.lo[1] == 0 && eb_hi[1] - 1 > ehi[1]) eys.push_back(eb_hi[1] - 1);
        for (int ez = elo[2]; ez <= ehi[2]; ++ez)
            for (int ey : eys)
                for (int ex = elo[0]; ex <= ehi[0]; ++ex) {
                    int16_t pos[81];
                    bool any_pivot = false;
                    for (int a = 0; a < 27; ++a) {
                        int x = 2 * ex + a % 3, y = B.wrap_y(2 * ey + (a / 3) % 3), z = 2 * ez + a / 9;
                        bool act = Builder::inside(A, x, y, z);
                        int64_t li = act ? B.lidx(x, y, z) : 0;
                        uint8_t mask = act ? B.node_comp_mask[li] : 0;
                        int f = act ? B.node_first[li] : -1;
                        int k = 0;
                        for (int c = 0; c < 3; ++c) {
                            int16_t v = -1;
                            if (mask & (1u << c)) {
                                int g = f + k;
                                ++k;
                                if (g >= s.first && g < s.first + s.p) {
                                    v = (int16_t)(g - s.first);
                                    any_pivot = true;
                                } else if (g >= s.first + s.p) {
                                    auto it = std::lower_bound(st.begin(), st.end(), g);
                                    if (it != st.end() && *it == g) v = (int16_t)(s.p + (it - st.begin()));
                                }
                            }
                            pos[3 * a + c] = v;
                        }
                    }
                    if (!any_pivot) continue;
                    int64_t e = (int64_t)ex + (int64_t)m.nx * ((int64_t)ey + (int64_t)m.ny * ez);
                    S.pair_elem.push_back((int)e);
                    S.pair_pos.insert(S.pair_pos.end(), pos, pos + 81);
                    ++s.n_elem_pairs;
                }
        if (s.p + s.q > 32767) fail(GL_ERR_INVALID_ARG, "symbolic: front larger than 32767 rows");
    }
}

}  // namespace gl
