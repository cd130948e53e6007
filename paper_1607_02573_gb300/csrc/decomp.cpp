// ORAS decomposition (Section 3) and the slot maps that drive assembly.
//
// * partition T_i: recursive coordinate bisection of tet centroids (the paper
//   uses SCOTCH/METIS; any partition is admissible): split along the axis of
//   largest centroid extent at floor(|T| p_left / p), p_left = p / 2, after
//   sorting by (centroid, tet id); or the caller's own tet -> part map;
// * overlap T_i^delta: delta times, add every tet sharing a vertex with the set;
// * partition of unity (Eq. chi): chi_i = 1 / (number of subdomains whose
//   T_j^0 contains the node) on the nodes of T_i^0, 0 elsewhere; D_i = chi_i
//   interpolated at edge midpoints / face centroids (Eq. algebPartUnity);
// * B_i = form restricted to T_i^delta + i k int (E x n).(v x n) on faces of
//   T_i^delta interior to the domain (k = k0 sqrt(eps_t), t the inside tet)
//   and on its physical impedance faces.
#include <algorithm>
#include <cmath>
#include <numeric>

#include "common.h"
#include "model.h"

namespace mwi {

void rcb_partition(const Topology& T, int nparts, std::vector<int32_t>& part) {
    const int64_t nt = T.nt;
    part.assign(nt, 0);
    std::vector<int32_t> ids(nt);
    std::iota(ids.begin(), ids.end(), 0);
    struct Rec {
        static void go(const std::vector<double>& cen, std::vector<int32_t>& part, int32_t* ids,
                       int64_t n, int p, int first) {
            if (p == 1) {
                for (int64_t i = 0; i < n; ++i) part[ids[i]] = first;
                return;
            }
            double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
            for (int64_t i = 0; i < n; ++i)
                for (int d = 0; d < 3; ++d) {
                    double v = cen[3 * (int64_t)ids[i] + d];
                    lo[d] = std::min(lo[d], v);
                    hi[d] = std::max(hi[d], v);
                }
            int ax = 0;
            double best = hi[0] - lo[0];
            for (int d = 1; d < 3; ++d)
                if (hi[d] - lo[d] > best) { best = hi[d] - lo[d]; ax = d; }
            std::sort(ids, ids + n, [&](int32_t a, int32_t b) {
                double va = cen[3 * (int64_t)a + ax], vb = cen[3 * (int64_t)b + ax];
                if (va != vb) return va < vb;
                return a < b;
            });
            int pl = p / 2;
            int64_t cut = (n * pl) / p;
            go(cen, part, ids, cut, pl, first);
            go(cen, part, ids + cut, n - cut, p - pl, first + pl);
        }
    };
    Rec::go(T.centroid, part, ids.data(), nt, nparts, 0);
}

// Sparse pattern + per-slot contribution lists for a set of rows.
// rows_glob: global DOF of each row (local numbering = position); g2l maps
// global -> local (-1 outside).  Elements are the tets in `tets` (ascending)
// then the face uses (ascending).
static void build_slots(const Topology& T, const std::vector<int32_t>& rows_glob,
                        const std::vector<int32_t>& g2l, const std::vector<int32_t>& tets,
                        const std::vector<uint8_t>* tet_in, const FaceUses& fu, int64_t fu_base,
                        SlotMatrix& S) {
    const int nl = T.nl, nlf = T.nlf;
    const int64_t n = (int64_t)rows_glob.size();
    S.nrows = n;
    S.row_ptr.assign(n + 1, 0);
    std::vector<std::vector<int32_t>> cols(n);
    std::vector<int32_t> buf;
    for (int64_t r = 0; r < n; ++r) {
        int32_t g = rows_glob[r];
        buf.clear();
        for (int32_t q = T.d2t_ptr[g]; q < T.d2t_ptr[g + 1]; ++q) {
            int32_t t = T.d2t[q] / nl;
            if (tet_in && !(*tet_in)[t]) continue;
            for (int j = 0; j < nl; ++j) {
                int32_t d = T.tet_dofs[(int64_t)nl * t + j];
                if (d < 0) continue;
                int32_t l = g2l[d];
                if (l >= 0) buf.push_back(l);
            }
        }
        std::sort(buf.begin(), buf.end());
        buf.erase(std::unique(buf.begin(), buf.end()), buf.end());
        cols[r] = buf;
        S.row_ptr[r + 1] = S.row_ptr[r] + (int64_t)buf.size();
    }
    const int64_t nnz = S.row_ptr[n];
    S.col.resize(nnz);
    for (int64_t r = 0; r < n; ++r)
        std::copy(cols[r].begin(), cols[r].end(), S.col.begin() + S.row_ptr[r]);
    cols.clear();
    cols.shrink_to_fit();
    auto find_slot = [&](int32_t r, int32_t c) -> int64_t {
        const int32_t* b = S.col.data() + S.row_ptr[r];
        const int32_t* e = S.col.data() + S.row_ptr[r + 1];
        const int32_t* it = std::lower_bound(b, e, c);
        if (it == e || *it != c) throw Error(MWI_EINVAL, "internal: slot not in pattern");
        return it - S.col.data();
    };
    // two passes: count, then fill in element order
    S.slot_ptr.assign(nnz + 1, 0);
    int loc[20];
    for (int pass = 0; pass < 2; ++pass) {
        std::vector<int64_t> fill;
        if (pass == 1) {
            for (int64_t s = 0; s < nnz; ++s) S.slot_ptr[s + 1] += S.slot_ptr[s];
            S.contrib.resize(S.slot_ptr[nnz]);
            fill.assign(S.slot_ptr.begin(), S.slot_ptr.end() - 1);
        }
        for (int32_t t : tets) {
            for (int i = 0; i < nl; ++i) {
                int32_t d = T.tet_dofs[(int64_t)nl * t + i];
                loc[i] = d >= 0 ? g2l[d] : -1;
            }
            for (int i = 0; i < nl; ++i) {
                if (loc[i] < 0) continue;
                for (int j = 0; j < nl; ++j) {
                    if (loc[j] < 0) continue;
                    int64_t s = find_slot(loc[i], loc[j]);
                    if (pass == 0) S.slot_ptr[s + 1]++;
                    else S.contrib[fill[s]++] = ((int64_t)t << 16) | pack_idx(i, j, nl);
                }
            }
        }
        for (size_t k = 0; k < fu.face.size(); ++k) {
            int32_t f = fu.face[k];
            for (int i = 0; i < nlf; ++i) {
                int32_t d = T.face_dofs[(int64_t)nlf * f + i];
                loc[i] = d >= 0 ? g2l[d] : -1;
            }
            for (int i = 0; i < nlf; ++i) {
                if (loc[i] < 0) continue;
                for (int j = 0; j < nlf; ++j) {
                    if (loc[j] < 0) continue;
                    int64_t s = find_slot(loc[i], loc[j]);
                    if (pass == 0) S.slot_ptr[s + 1]++;
                    else
                        S.contrib[fill[s]++] =
                            kFaceFlag | ((int64_t)(fu_base + (int64_t)k) << 16) | pack_idx(i, j, nlf);
                }
            }
        }
    }
}

void build_global_slots(const Topology& T, SlotMatrix& A, FaceUses& fu) {
    std::vector<int32_t> rows(T.ndof), g2l(T.ndof);
    std::iota(rows.begin(), rows.end(), 0);
    std::iota(g2l.begin(), g2l.end(), 0);
    std::vector<int32_t> tets(T.nt);
    std::iota(tets.begin(), tets.end(), 0);
    fu.face.clear();
    fu.tet.clear();
    for (int64_t f = 0; f < T.nf; ++f)
        if (T.face_tag[f] == TAG_IMPEDANCE) {
            fu.face.push_back((int32_t)f);
            fu.tet.push_back(T.face_tets[2 * f]);
        }
    build_slots(T, rows, g2l, tets, nullptr, fu, 0, A);
}

void build_decomposition(const Topology& T, const int32_t* part_in, int n_sub, int overlap,
                         int nd_leaf, Decomposition& D) {
    MWI_REQUIRE(n_sub >= 1 && n_sub <= 65536, MWI_EINVAL, "n_sub out of range");
    MWI_REQUIRE(overlap >= 0 && overlap <= 8, MWI_EINVAL, "overlap out of range");
    const int64_t nt = T.nt, nv = T.nv;
    D.n_sub = n_sub;
    D.overlap = overlap;
    D.nd_leaf = std::max(8, nd_leaf);
    if (part_in) {
        D.part.assign(part_in, part_in + nt);
        for (int32_t p : D.part) MWI_REQUIRE(p >= 0 && p < n_sub, MWI_EINVAL, "part value out of range");
    } else {
        rcb_partition(T, n_sub, D.part);
    }
    std::vector<std::vector<int32_t>> T0(n_sub);
    for (int64_t t = 0; t < nt; ++t) T0[D.part[t]].push_back((int32_t)t);
    for (int i = 0; i < n_sub; ++i) MWI_REQUIRE(!T0[i].empty(), MWI_EINVAL, "empty subdomain");

    // node counts for the partition of unity
    std::vector<int32_t> cnt(nv, 0), stamp(nv, -1);
    for (int i = 0; i < n_sub; ++i)
        for (int32_t t : T0[i])
            for (int k = 0; k < 4; ++k) {
                int32_t v = T.tv[4 * (int64_t)t + k];
                if (stamp[v] != i) { stamp[v] = i; cnt[v]++; }
            }

    D.sub_off.assign(n_sub + 1, 0);
    D.loc2glob.clear();
    D.dweight.clear();
    D.B = SlotMatrix();
    D.B.row_ptr.assign(1, 0);
    D.B.slot_ptr.assign(1, 0);
    D.B_faces = FaceUses();
    D.fronts.clear();
    D.urows.clear();
    D.urel.clear();
    D.amap_slot.clear();
    D.amap_pos.clear();
    D.amap_front_ptr.assign(1, 0);
    D.child_ptr.clear();
    D.child.clear();
    D.ws_entries = 0;
    D.upd_rows = 0;
    D.factor_entries = 0;
    D.factor_flops = 0;
    D.max_front = 0;

    std::vector<uint8_t> tet_in(nt, 0), vmark(nv, 0);
    std::vector<int32_t> g2l(T.ndof, -1);
    std::vector<double> chi(nv, 0.0);
    std::vector<std::vector<int32_t>> front_children;

    for (int i = 0; i < n_sub; ++i) {
        // T_i^delta
        std::vector<int32_t> cur = T0[i];
        for (int32_t t : cur) tet_in[t] = 1;
        for (int d = 0; d < overlap; ++d) {
            std::vector<int32_t> touched;
            for (int32_t t : cur)
                for (int k = 0; k < 4; ++k) {
                    int32_t v = T.tv[4 * (int64_t)t + k];
                    if (!vmark[v]) { vmark[v] = 1; touched.push_back(v); }
                }
            std::vector<int32_t> nxt = cur;
            for (int32_t v : touched)
                for (int32_t q = T.v2t_ptr[v]; q < T.v2t_ptr[v + 1]; ++q) {
                    int32_t t = T.v2t[q];
                    if (!tet_in[t]) { tet_in[t] = 1; nxt.push_back(t); }
                }
            for (int32_t v : touched) vmark[v] = 0;
            cur.swap(nxt);
        }
        std::sort(cur.begin(), cur.end());
        // chi_i on the nodes of T_i^0
        std::vector<int32_t> nodes0;
        for (int32_t t : T0[i])
            for (int k = 0; k < 4; ++k) {
                int32_t v = T.tv[4 * (int64_t)t + k];
                if (chi[v] == 0.0) { chi[v] = 1.0 / (double)cnt[v]; nodes0.push_back(v); }
            }
        // local DOFs (natural order = ascending global id)
        std::vector<int32_t> dofs;
        for (int32_t t : cur)
            for (int j = 0; j < T.nl; ++j) {
                int32_t d = T.tet_dofs[(int64_t)T.nl * t + j];
                if (d >= 0 && g2l[d] < 0) { g2l[d] = 0; dofs.push_back(d); }
            }
        std::sort(dofs.begin(), dofs.end());
        for (size_t l = 0; l < dofs.size(); ++l) g2l[dofs[l]] = (int32_t)l;
        MWI_REQUIRE(!dofs.empty(), MWI_EINVAL, "subdomain without DOFs");

        // nested-dissection ordering of the local DOFs (graph of B_i, natural numbering)
        std::vector<int32_t> nd_order;  // nd_order[k] = natural local index at ND position k
        const size_t front_first = D.fronts.size();
        {
            std::vector<std::vector<int32_t>> adj(dofs.size());
            std::vector<int32_t> buf;
            for (size_t r = 0; r < dofs.size(); ++r) {
                int32_t g = dofs[r];
                buf.clear();
                for (int32_t q = T.d2t_ptr[g]; q < T.d2t_ptr[g + 1]; ++q) {
                    int32_t t = T.d2t[q] / T.nl;
                    if (!tet_in[t]) continue;
                    for (int j = 0; j < T.nl; ++j) {
                        int32_t d = T.tet_dofs[(int64_t)T.nl * t + j];
                        if (d >= 0 && d != g) buf.push_back(g2l[d]);
                    }
                }
                std::sort(buf.begin(), buf.end());
                buf.erase(std::unique(buf.begin(), buf.end()), buf.end());
                adj[r] = buf;
            }
            symbolic_subdomain(T, D, i, dofs, adj, nd_order);
        }
        // local rows in ND order
        std::vector<int32_t> rows_nd(dofs.size());
        for (size_t k = 0; k < dofs.size(); ++k) rows_nd[k] = dofs[nd_order[k]];
        for (size_t k = 0; k < rows_nd.size(); ++k) g2l[rows_nd[k]] = (int32_t)k;
        const int64_t base = D.sub_off[i];
        D.sub_off[i + 1] = base + (int64_t)rows_nd.size();
        for (int32_t g : rows_nd) {
            D.loc2glob.push_back(g);
            double s = 0.0;
            int nvx = 0;
            for (int k = 0; k < 3; ++k) {
                int64_t v = T.dof_verts[3 * (int64_t)g + k];
                if (v >= 0) { s += chi[v]; nvx++; }
            }
            D.dweight.push_back(s / (double)nvx);
        }

        // face uses of B_i: faces of T_i^delta tets on its boundary (not PEC)
        FaceUses fu;
        for (int32_t t : cur)
            for (int lf = 0; lf < 4; ++lf) {
                int32_t f = T.tet_faces[4 * (int64_t)t + lf];
                if (T.face_tag[f] == TAG_PEC) continue;
                int32_t a = T.face_tets[2 * f], b = T.face_tets[2 * f + 1];
                int32_t other = (a == t) ? b : a;
                bool boundary = other < 0 || !tet_in[other];
                if (!boundary) continue;
                fu.face.push_back(f);
                fu.tet.push_back(t);
            }
        SlotMatrix Bi;
        build_slots(T, rows_nd, g2l, cur, &tet_in, fu, (int64_t)D.B_faces.face.size(), Bi);
        // append B_i to the block-diagonal B (columns stay local to the subdomain)
        const int64_t slot_base = (int64_t)D.B.col.size();
        const int64_t contrib_base = (int64_t)D.B.contrib.size();
        for (int64_t r = 0; r < Bi.nrows; ++r) D.B.row_ptr.push_back(slot_base + Bi.row_ptr[r + 1]);
        D.B.col.insert(D.B.col.end(), Bi.col.begin(), Bi.col.end());
        for (int64_t s = 0; s < (int64_t)Bi.col.size(); ++s)
            D.B.slot_ptr.push_back(contrib_base + Bi.slot_ptr[s + 1]);
        D.B.contrib.insert(D.B.contrib.end(), Bi.contrib.begin(), Bi.contrib.end());
        D.B_faces.face.insert(D.B_faces.face.end(), fu.face.begin(), fu.face.end());
        D.B_faces.tet.insert(D.B_faces.tet.end(), fu.tet.begin(), fu.tet.end());

        // front assembly map: pivot row v of front s, entries (v, w) with w >= v
        for (size_t fi = front_first; fi < D.fronts.size(); ++fi) {
            Front& F = D.fronts[fi];
            const int32_t fsz = F.p + F.u;
            const int32_t* U = D.urows.data() + F.u_off;
            for (int32_t c = 0; c < F.p; ++c) {
                int32_t v = F.start + c;
                for (int64_t q = Bi.row_ptr[v]; q < Bi.row_ptr[v + 1]; ++q) {
                    int32_t w = Bi.col[q];
                    if (w < v) continue;
                    int32_t r;
                    if (w < F.start + F.p) r = w - F.start;
                    else {
                        const int32_t* it = std::lower_bound(U, U + F.u, w);
                        MWI_REQUIRE(it != U + F.u && *it == w, MWI_EINVAL, "internal: entry outside front");
                        r = F.p + (int32_t)(it - U);
                    }
                    D.amap_slot.push_back(slot_base + q);
                    D.amap_pos.push_back(F.f_off + (int64_t)c * fsz + r);
                }
            }
            D.amap_front_ptr.push_back((int64_t)D.amap_slot.size());
        }

        // reset per-subdomain marks
        for (int32_t t : cur) tet_in[t] = 0;
        for (int32_t v : nodes0) chi[v] = 0.0;
        for (int32_t g : rows_nd) g2l[g] = -1;
    }
    D.B.nrows = D.sub_off[n_sub];

    // scatter lists R_i^T D_i: rows with D > 0 per global DOF, subdomains ascending
    const int64_t nloc = D.sub_off[n_sub];
    D.own_ptr.assign(T.ndof + 1, 0);
    for (int64_t r = 0; r < nloc; ++r)
        if (D.dweight[r] > 0.0) D.own_ptr[D.loc2glob[r] + 1]++;
    for (int64_t g = 0; g < T.ndof; ++g) D.own_ptr[g + 1] += D.own_ptr[g];
    D.own_row.resize(D.own_ptr[T.ndof]);
    D.own_w.resize(D.own_ptr[T.ndof]);
    {
        std::vector<int64_t> fill(D.own_ptr.begin(), D.own_ptr.end() - 1);
        for (int64_t r = 0; r < nloc; ++r)
            if (D.dweight[r] > 0.0) {
                int64_t k = fill[D.loc2glob[r]]++;
                D.own_row[k] = (int32_t)r;
                D.own_w[k] = D.dweight[r];
            }
    }
    for (int64_t g = 0; g < T.ndof; ++g)
        MWI_REQUIRE(D.own_ptr[g + 1] > D.own_ptr[g], MWI_EINVAL, "internal: DOF without owner");

    // fronts grouped by tree depth (deepest first) and child lists
    int maxd = 0;
    for (const Front& F : D.fronts) maxd = std::max(maxd, (int)F.level);
    D.n_levels = maxd + 1;
    D.level_ptr.assign(D.n_levels + 1, 0);
    D.level_fronts.clear();
    for (int d = maxd; d >= 0; --d) {
        for (size_t k = 0; k < D.fronts.size(); ++k)
            if (D.fronts[k].level == d) D.level_fronts.push_back((int32_t)k);
        D.level_ptr[maxd - d + 1] = (int32_t)D.level_fronts.size();
    }
    const int64_t nfr = (int64_t)D.fronts.size();
    D.child_ptr.assign(nfr + 1, 0);
    for (const Front& F : D.fronts)
        if (F.parent >= 0) D.child_ptr[F.parent + 1]++;
    for (int64_t k = 0; k < nfr; ++k) D.child_ptr[k + 1] += D.child_ptr[k];
    D.child.resize(D.child_ptr[nfr]);
    {
        std::vector<int32_t> fill(D.child_ptr.begin(), D.child_ptr.end() - 1);
        for (int64_t k = 0; k < nfr; ++k)
            if (D.fronts[k].parent >= 0) D.child[fill[D.fronts[k].parent]++] = (int32_t)k;
    }
}

}  // namespace mwi
