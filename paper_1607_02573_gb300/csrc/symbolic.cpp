// Symbolic analysis of one subdomain operator B_i for the batched multifrontal
// LDL^T factorisation.  The ordering is a geometric nested dissection of the
// DOF positions: split the set at the median along its longest extent, take
// as separator the smaller of the two one-sided boundaries, recurse on both
// halves, and number the separator after them.  The dissection tree is the
// assembly tree: every separator (or leaf) is a supernode whose pivots are
// contiguous in the new order, and its front holds the pivots plus the update
// set U_s of ancestor DOFs coupled to its subtree.  Fronts are dense.
#include <algorithm>
#include <numeric>

#include "common.h"
#include "model.h"

namespace mwi {

namespace {

struct Node {
    std::vector<int32_t> piv;   // natural indices
    int32_t parent = -1;
    int32_t depth = 0;
    int32_t start = 0;          // ND index of first pivot
    std::vector<int32_t> kids;
    std::vector<int32_t> U;     // ND indices, sorted
};

struct Ctx {
    const Topology* T;
    const std::vector<int32_t>* rows;
    const std::vector<std::vector<int32_t>>* adj;
    int leaf;
    std::vector<Node> nodes;
    std::vector<int32_t> nd_pos;   // natural -> ND position
    std::vector<int8_t> side;      // scratch: -1 outside, 0 left, 1 right
    int32_t next = 0;

    double coord(int32_t v, int ax) const {
        return T->dof_pos[3 * (int64_t)(*rows)[v] + ax];
    }

    int32_t make_node(std::vector<int32_t>&& piv, int depth) {
        Node nd;
        nd.piv = std::move(piv);
        nd.depth = depth;
        nd.start = next;
        for (int32_t v : nd.piv) nd_pos[v] = next++;
        nodes.push_back(std::move(nd));
        return (int32_t)nodes.size() - 1;
    }

    int32_t rec(std::vector<int32_t>& set, int depth) {
        if ((int)set.size() <= leaf) return make_node(std::move(set), depth);
        double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
        for (int32_t v : set)
            for (int d = 0; d < 3; ++d) {
                lo[d] = std::min(lo[d], coord(v, d));
                hi[d] = std::max(hi[d], coord(v, d));
            }
        int ax = 0;
        for (int d = 1; d < 3; ++d)
            if (hi[d] - lo[d] > hi[ax] - lo[ax]) ax = d;
        std::sort(set.begin(), set.end(), [&](int32_t a, int32_t b) {
            double ca = coord(a, ax), cb = coord(b, ax);
            if (ca != cb) return ca < cb;
            return a < b;
        });
        const size_t half = set.size() / 2;
        for (size_t k = 0; k < set.size(); ++k) side[set[k]] = k < half ? 0 : 1;
        std::vector<int32_t> sepL, sepR;
        for (size_t k = 0; k < set.size(); ++k) {
            int32_t v = set[k];
            for (int32_t w : (*adj)[v])
                if (side[w] >= 0 && side[w] != side[v]) {
                    (side[v] == 0 ? sepL : sepR).push_back(v);
                    break;
                }
        }
        std::vector<int32_t>& sep = (sepR.size() < sepL.size()) ? sepR : sepL;
        if (sep.empty()) sep.push_back(set[half - 1]);  // disconnected halves
        for (int32_t v : sep) side[v] = 2;
        std::vector<int32_t> L, R;
        for (int32_t v : set) {
            if (side[v] == 0) L.push_back(v);
            else if (side[v] == 1) R.push_back(v);
        }
        for (int32_t v : set) side[v] = -1;
        std::vector<int32_t> sep_copy = sep;
        std::vector<int32_t> kids;
        if (!L.empty()) kids.push_back(rec(L, depth + 1));
        if (!R.empty()) kids.push_back(rec(R, depth + 1));
        int32_t id = make_node(std::move(sep_copy), depth);
        for (int32_t c : kids) {
            nodes[c].parent = id;
            nodes[id].kids.push_back(c);
        }
        return id;
    }
};

}  // namespace

void symbolic_subdomain(const Topology& T, int nd_leaf, const std::vector<int32_t>& rows_glob,
                        const std::vector<std::vector<int32_t>>& adj, LocalSymbolic& out) {
    const int32_t n = (int32_t)rows_glob.size();
    Ctx C;
    C.T = &T;
    C.rows = &rows_glob;
    C.adj = &adj;
    C.leaf = nd_leaf;
    C.nd_pos.assign(n, -1);
    C.side.assign(n, -1);
    std::vector<int32_t> all(n);
    std::iota(all.begin(), all.end(), 0);
    C.rec(all, 0);
    out.nd_order.assign(n, -1);
    for (int32_t v = 0; v < n; ++v) out.nd_order[C.nd_pos[v]] = v;

    // update sets, children before parents (creation order is a postorder)
    std::vector<int32_t> buf;
    for (Node& s : C.nodes) {
        const int32_t end = s.start + (int32_t)s.piv.size();
        buf.clear();
        for (int32_t v : s.piv)
            for (int32_t w : adj[v]) {
                const int32_t x = C.nd_pos[w];
                if (x >= end) buf.push_back(x);
            }
        for (int32_t c : s.kids)
            for (int32_t x : C.nodes[c].U)
                if (x >= end) buf.push_back(x);
        std::sort(buf.begin(), buf.end());
        buf.erase(std::unique(buf.begin(), buf.end()), buf.end());
        s.U = buf;
    }
    out.fronts.clear();
    out.urows.clear();
    out.flops = 0;
    for (const Node& s : C.nodes) {
        LocalFront F;
        F.start = s.start;
        F.p = (int32_t)s.piv.size();
        F.u = (int32_t)s.U.size();
        F.parent = s.parent;
        F.level = s.depth;
        F.u_off = (int64_t)out.urows.size();
        out.urows.insert(out.urows.end(), s.U.begin(), s.U.end());
        const int64_t f = (int64_t)F.p + F.u;
        for (int64_t j = 0; j < F.p; ++j) {
            const double r = (double)(f - j - 1);
            out.flops += 8.0 * (r + 0.5 * r * (r + 1.0));
        }
        out.fronts.push_back(F);
    }
    // relative positions of every child's update rows in its parent's front
    out.urel.assign(out.urows.size(), -1);
    for (size_t k = 0; k < C.nodes.size(); ++k) {
        const Node& s = C.nodes[k];
        if (s.parent < 0) {
            MWI_REQUIRE(s.U.empty(), MWI_EINVAL, "internal: root front with update rows");
            continue;
        }
        const Node& P = C.nodes[s.parent];
        const int32_t pend = P.start + (int32_t)P.piv.size();
        for (size_t j = 0; j < s.U.size(); ++j) {
            const int32_t x = s.U[j];
            int32_t pos;
            if (x < pend) {
                MWI_REQUIRE(x >= P.start, MWI_EINVAL, "internal: update row below parent pivots");
                pos = x - P.start;
            } else {
                auto it = std::lower_bound(P.U.begin(), P.U.end(), x);
                MWI_REQUIRE(it != P.U.end() && *it == x, MWI_EINVAL, "internal: update row not in parent");
                pos = (int32_t)P.piv.size() + (int32_t)(it - P.U.begin());
            }
            out.urel[out.fronts[k].u_off + j] = pos;
        }
    }
}

}  // namespace mwi
