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
#include <mutex>
#include <numeric>

#include "common.h"
#include "model.h"
#include "parallel.h"

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
// global -> local (-1 outside); tet_in (optional) restricts the tets.
// Every slot (r, c) lists its contributions in a fixed order: the tets that
// hold both DOFs in ascending tet id, then the face uses in ascending order.
// Each row is built by its own thread ("pull"), so the order does not depend
// on the scheduling.
static void build_slots(const Topology& T, const std::vector<int32_t>& rows_glob,
                        const std::vector<int32_t>& g2l, const std::vector<uint8_t>* tet_in, const FaceUses& fu,
                        int64_t fu_base, SlotMatrix& S, bool threaded) {
    const int nl = T.nl, nlf = T.nlf;
    const int64_t n = (int64_t)rows_glob.size();
    S.nrows = n;
    // DOF -> face uses (ascending use index) for the rows of this matrix
    std::vector<int64_t> fptr(n + 1, 0);
    std::vector<int32_t> fuse;
    for (size_t k = 0; k < fu.face.size(); ++k)
        for (int i = 0; i < nlf; ++i) {
            const int32_t d = T.face_dofs[(int64_t)nlf * fu.face[k] + i];
            if (d >= 0 && g2l[d] >= 0) fptr[g2l[d] + 1]++;
        }
    for (int64_t r = 0; r < n; ++r) fptr[r + 1] += fptr[r];
    fuse.resize(fptr[n]);
    {
        std::vector<int64_t> fill(fptr.begin(), fptr.end() - 1);
        for (size_t k = 0; k < fu.face.size(); ++k)
            for (int i = 0; i < nlf; ++i) {
                const int32_t d = T.face_dofs[(int64_t)nlf * fu.face[k] + i];
                if (d >= 0 && g2l[d] >= 0) fuse[fill[g2l[d]]++] = (int32_t)k;
            }
    }
    auto run = [&](int64_t count, auto&& fn) {
        if (threaded) parallel_for(count, 256, fn);
        else for (int64_t i = 0; i < count; ++i) fn(i, 0);
    };
    // pattern
    std::vector<std::vector<int32_t>> cols(n);
    run(n, [&](int64_t r, int) {
        const int32_t g = rows_glob[r];
        std::vector<int32_t>& buf = cols[r];
        for (int32_t q = T.d2t_ptr[g]; q < T.d2t_ptr[g + 1]; ++q) {
            const int32_t t = T.d2t[q] / nl;
            if (tet_in && !(*tet_in)[t]) continue;
            for (int j = 0; j < nl; ++j) {
                const int32_t d = T.tet_dofs[(int64_t)nl * t + j];
                if (d >= 0 && g2l[d] >= 0) buf.push_back(g2l[d]);
            }
        }
        std::sort(buf.begin(), buf.end());
        buf.erase(std::unique(buf.begin(), buf.end()), buf.end());
    });
    S.row_ptr.assign(n + 1, 0);
    for (int64_t r = 0; r < n; ++r) S.row_ptr[r + 1] = S.row_ptr[r] + (int64_t)cols[r].size();
    const int64_t nnz = S.row_ptr[n];
    S.col.resize(nnz);
    run(n, [&](int64_t r, int) {
        std::copy(cols[r].begin(), cols[r].end(), S.col.begin() + S.row_ptr[r]);
        std::vector<int32_t>().swap(cols[r]);
    });
    auto find_slot = [&](int64_t r, int32_t c) -> int64_t {
        const int32_t* b = S.col.data() + S.row_ptr[r];
        const int32_t* e = S.col.data() + S.row_ptr[r + 1];
        const int32_t* it = std::lower_bound(b, e, c);
        if (it == e || *it != c) throw Error(MWI_EINVAL, "internal: slot not in pattern");
        return it - S.col.data();
    };
    // visit the contributions of row r in their fixed order
    auto visit = [&](int64_t r, auto&& emit) {
        const int32_t g = rows_glob[r];
        for (int32_t q = T.d2t_ptr[g]; q < T.d2t_ptr[g + 1]; ++q) {
            const int32_t t = T.d2t[q] / nl, li = T.d2t[q] % nl;
            if (tet_in && !(*tet_in)[t]) continue;
            for (int j = 0; j < nl; ++j) {
                const int32_t d = T.tet_dofs[(int64_t)nl * t + j];
                if (d < 0 || g2l[d] < 0) continue;
                emit(find_slot(r, g2l[d]), ((int64_t)t << 16) | pack_idx(li, j, nl));
            }
        }
        for (int64_t q = fptr[r]; q < fptr[r + 1]; ++q) {
            const int32_t k = fuse[q];
            const int32_t f = fu.face[k];
            int fi = -1;
            for (int i = 0; i < nlf; ++i)
                if (T.face_dofs[(int64_t)nlf * f + i] == g) fi = i;
            for (int j = 0; j < nlf; ++j) {
                const int32_t d = T.face_dofs[(int64_t)nlf * f + j];
                if (d < 0 || g2l[d] < 0) continue;
                emit(find_slot(r, g2l[d]), kFaceFlag | ((int64_t)(fu_base + k) << 16) | pack_idx(fi, j, nlf));
            }
        }
    };
    S.slot_ptr.assign(nnz + 1, 0);
    run(n, [&](int64_t r, int) { visit(r, [&](int64_t sl, int64_t) { S.slot_ptr[sl + 1]++; }); });
    for (int64_t q = 0; q < nnz; ++q) S.slot_ptr[q + 1] += S.slot_ptr[q];
    S.contrib.resize(S.slot_ptr[nnz]);
    std::vector<int32_t> used(nnz, 0);
    run(n, [&](int64_t r, int) {
        visit(r, [&](int64_t sl, int64_t c) { S.contrib[S.slot_ptr[sl] + used[sl]++] = c; });
    });
}

void build_global_slots(const Topology& T, SlotMatrix& A, FaceUses& fu) {
    std::vector<int32_t> rows(T.ndof), g2l(T.ndof);
    std::iota(rows.begin(), rows.end(), 0);
    std::iota(g2l.begin(), g2l.end(), 0);
    fu.face.clear();
    fu.tet.clear();
    for (int64_t f = 0; f < T.nf; ++f)
        if (T.face_tag[f] == TAG_IMPEDANCE) {
            fu.face.push_back((int32_t)f);
            fu.tet.push_back(T.face_tets[2 * f]);
        }
    build_slots(T, rows, g2l, nullptr, fu, 0, A, true);
}

namespace {

// Everything one subdomain contributes, computed independently of the others.
struct SubWork {
    std::vector<int32_t> rows_nd;   // global DOFs in ND order
    std::vector<double> dw;         // D_i weights
    FaceUses fu;                    // impedance face uses of B_i
    SlotMatrix Bi;                  // B_i pattern and slot maps (local ND numbering)
    LocalSymbolic sym;              // fronts of the subdomain
    std::vector<int64_t> am_slot;   // assembly map: local slot of B_i
    std::vector<int64_t> am_pos;    // position inside the front: col * f + row
    std::vector<int64_t> am_ptr;    // per local front
};

struct Scratch {
    std::vector<uint8_t> tet_in, vmark, node0;
    std::vector<int32_t> g2l;
};

void subdomain_work(const Topology& T, const std::vector<int32_t>& T0, const std::vector<int32_t>& cnt, int overlap,
                    int nd_leaf, Scratch& sc, SubWork& W) {
    std::vector<uint8_t>& tet_in = sc.tet_in;
    std::vector<uint8_t>& vmark = sc.vmark;
    std::vector<uint8_t>& node0 = sc.node0;
    std::vector<int32_t>& g2l = sc.g2l;
    // T_i^delta
    std::vector<int32_t> cur = T0;
    for (int32_t t : cur) tet_in[t] = 1;
    for (int d = 0; d < overlap; ++d) {
        std::vector<int32_t> touched;
        for (int32_t t : cur)
            for (int k = 0; k < 4; ++k) {
                const int32_t v = T.tv[4 * (int64_t)t + k];
                if (!vmark[v]) { vmark[v] = 1; touched.push_back(v); }
            }
        std::vector<int32_t> nxt = cur;
        for (int32_t v : touched)
            for (int32_t q = T.v2t_ptr[v]; q < T.v2t_ptr[v + 1]; ++q) {
                const int32_t t = T.v2t[q];
                if (!tet_in[t]) { tet_in[t] = 1; nxt.push_back(t); }
            }
        for (int32_t v : touched) vmark[v] = 0;
        cur.swap(nxt);
    }
    std::sort(cur.begin(), cur.end());
    // nodes of T_i^0 (chi_i = 1 / cnt there)
    std::vector<int32_t> nodes0;
    for (int32_t t : T0)
        for (int k = 0; k < 4; ++k) {
            const int32_t v = T.tv[4 * (int64_t)t + k];
            if (!node0[v]) { node0[v] = 1; nodes0.push_back(v); }
        }
    // local DOFs (natural order = ascending global id)
    std::vector<int32_t> dofs;
    for (int32_t t : cur)
        for (int j = 0; j < T.nl; ++j) {
            const int32_t d = T.tet_dofs[(int64_t)T.nl * t + j];
            if (d >= 0 && g2l[d] < 0) { g2l[d] = 0; dofs.push_back(d); }
        }
    std::sort(dofs.begin(), dofs.end());
    for (size_t l = 0; l < dofs.size(); ++l) g2l[dofs[l]] = (int32_t)l;
    MWI_REQUIRE(!dofs.empty(), MWI_EINVAL, "subdomain without DOFs");
    // nested-dissection ordering on the graph of B_i (natural numbering)
    {
        std::vector<std::vector<int32_t>> adj(dofs.size());
        for (size_t r = 0; r < dofs.size(); ++r) {
            const int32_t g = dofs[r];
            std::vector<int32_t>& buf = adj[r];
            for (int32_t q = T.d2t_ptr[g]; q < T.d2t_ptr[g + 1]; ++q) {
                const int32_t t = T.d2t[q] / T.nl;
                if (!tet_in[t]) continue;
                for (int j = 0; j < T.nl; ++j) {
                    const int32_t d = T.tet_dofs[(int64_t)T.nl * t + j];
                    if (d >= 0 && d != g) buf.push_back(g2l[d]);
                }
            }
            std::sort(buf.begin(), buf.end());
            buf.erase(std::unique(buf.begin(), buf.end()), buf.end());
        }
        symbolic_subdomain(T, nd_leaf, dofs, adj, W.sym);
    }
    W.rows_nd.resize(dofs.size());
    for (size_t k = 0; k < dofs.size(); ++k) W.rows_nd[k] = dofs[W.sym.nd_order[k]];
    for (size_t k = 0; k < W.rows_nd.size(); ++k) g2l[W.rows_nd[k]] = (int32_t)k;
    W.dw.resize(W.rows_nd.size());
    for (size_t k = 0; k < W.rows_nd.size(); ++k) {
        const int32_t g = W.rows_nd[k];
        double s = 0.0;
        int nvx = 0;
        for (int q = 0; q < 3; ++q) {
            const int64_t v = T.dof_verts[3 * (int64_t)g + q];
            if (v >= 0) {
                s += node0[v] ? 1.0 / (double)cnt[v] : 0.0;
                nvx++;
            }
        }
        W.dw[k] = s / (double)nvx;
    }
    // face uses: faces of T_i^delta tets on its boundary (not PEC)
    for (int32_t t : cur)
        for (int lf = 0; lf < 4; ++lf) {
            const int32_t f = T.tet_faces[4 * (int64_t)t + lf];
            if (T.face_tag[f] == TAG_PEC) continue;
            const int32_t a = T.face_tets[2 * f], b = T.face_tets[2 * f + 1];
            const int32_t other = (a == t) ? b : a;
            if (other >= 0 && tet_in[other]) continue;
            W.fu.face.push_back(f);
            W.fu.tet.push_back(t);
        }
    build_slots(T, W.rows_nd, g2l, &tet_in, W.fu, 0, W.Bi, false);
    // front assembly map: pivot row v of front s, entries (v, w) with w >= v
    W.am_ptr.assign(1, 0);
    for (const LocalFront& F : W.sym.fronts) {
        const int32_t fsz = F.p + F.u;
        const int32_t* U = W.sym.urows.data() + F.u_off;
        for (int32_t c = 0; c < F.p; ++c) {
            const int32_t v = F.start + c;
            for (int64_t q = W.Bi.row_ptr[v]; q < W.Bi.row_ptr[v + 1]; ++q) {
                const int32_t w = W.Bi.col[q];
                if (w < v) continue;
                int32_t r;
                if (w < F.start + F.p) r = w - F.start;
                else {
                    const int32_t* it = std::lower_bound(U, U + F.u, w);
                    MWI_REQUIRE(it != U + F.u && *it == w, MWI_EINVAL, "internal: entry outside front");
                    r = F.p + (int32_t)(it - U);
                }
                W.am_slot.push_back(q);
                W.am_pos.push_back((int64_t)c * fsz + r);
            }
        }
        W.am_ptr.push_back((int64_t)W.am_slot.size());
    }
    // reset marks
    for (int32_t t : cur) tet_in[t] = 0;
    for (int32_t v : nodes0) node0[v] = 0;
    for (int32_t g : W.rows_nd) g2l[g] = -1;
}

}  // namespace

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
                const int32_t v = T.tv[4 * (int64_t)t + k];
                if (stamp[v] != i) { stamp[v] = i; cnt[v]++; }
            }

    // independent per-subdomain work, one scratch set per worker thread
    std::vector<SubWork> work(n_sub);
    std::vector<Scratch> scratch(setup_threads());
    std::mutex smu;
    parallel_for(n_sub, 1, [&](int64_t i, int w) {
        Scratch& sc = scratch[w];
        if (sc.tet_in.empty()) {
            sc.tet_in.assign(nt, 0);
            sc.vmark.assign(nv, 0);
            sc.node0.assign(nv, 0);
            sc.g2l.assign(T.ndof, -1);
        }
        subdomain_work(T, T0[i], cnt, overlap, D.nd_leaf, sc, work[i]);
    });
    (void)smu;

    // concatenate in subdomain order
    D.sub_off.assign(n_sub + 1, 0);
    D.loc2glob.clear();
    D.dweight.clear();
    D.B = SlotMatrix();
    D.B.row_ptr.assign(1, 0);
    D.B.slot_ptr.assign(1, 0);
    D.B_faces = FaceUses();
    D.fu_off.assign(n_sub + 1, 0);
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
    for (int i = 0; i < n_sub; ++i) {
        SubWork& W = work[i];
        D.sub_off[i + 1] = D.sub_off[i] + (int64_t)W.rows_nd.size();
        D.loc2glob.insert(D.loc2glob.end(), W.rows_nd.begin(), W.rows_nd.end());
        D.dweight.insert(D.dweight.end(), W.dw.begin(), W.dw.end());
        const int64_t slot_base = (int64_t)D.B.col.size();
        const int64_t contrib_base = (int64_t)D.B.contrib.size();
        const int64_t fu_base = (int64_t)D.B_faces.face.size();
        for (int64_t r = 0; r < W.Bi.nrows; ++r) D.B.row_ptr.push_back(slot_base + W.Bi.row_ptr[r + 1]);
        D.B.col.insert(D.B.col.end(), W.Bi.col.begin(), W.Bi.col.end());
        for (int64_t q = 0; q < (int64_t)W.Bi.col.size(); ++q)
            D.B.slot_ptr.push_back(contrib_base + W.Bi.slot_ptr[q + 1]);
        for (int64_t c : W.Bi.contrib) {
            if (c & kFaceFlag) {
                const int64_t u = (c & (kFaceFlag - 1)) >> 16;
                c = kFaceFlag | ((u + fu_base) << 16) | (c & 0xffff);
            }
            D.B.contrib.push_back(c);
        }
        D.B_faces.face.insert(D.B_faces.face.end(), W.fu.face.begin(), W.fu.face.end());
        D.B_faces.tet.insert(D.B_faces.tet.end(), W.fu.tet.begin(), W.fu.tet.end());
        D.fu_off[i + 1] = (int64_t)D.B_faces.face.size();
        const int32_t front_base = (int32_t)D.fronts.size();
        for (size_t k = 0; k < W.sym.fronts.size(); ++k) {
            const LocalFront& L = W.sym.fronts[k];
            Front F;
            F.sub = i;
            F.start = L.start;
            F.p = L.p;
            F.u = L.u;
            F.parent = L.parent >= 0 ? front_base + L.parent : -1;
            F.level = L.level;
            const int64_t f = (int64_t)F.p + F.u;
            F.f_off = D.ws_entries;
            D.ws_entries += f * F.p;
            F.sch_off = 0;
            F.u_off = (int64_t)D.urows.size() + L.u_off;
            F.upd_row = D.upd_rows;
            D.upd_rows += F.u;
            D.factor_entries += f * F.p;
            D.max_front = std::max<int32_t>(D.max_front, (int32_t)f);
            for (int64_t q = W.am_ptr[k]; q < W.am_ptr[k + 1]; ++q) {
                D.amap_slot.push_back(slot_base + W.am_slot[q]);
                D.amap_pos.push_back(F.f_off + W.am_pos[q]);
            }
            D.amap_front_ptr.push_back((int64_t)D.amap_slot.size());
            D.fronts.push_back(F);
        }
        D.urows.insert(D.urows.end(), W.sym.urows.begin(), W.sym.urows.end());
        D.urel.insert(D.urel.end(), W.sym.urel.begin(), W.sym.urel.end());
        D.factor_flops += W.sym.flops;
        W = SubWork();
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
    // Schur blocks live in two transient buffers, even and odd levels (a
    // level's blocks are consumed by the next level's assembly)
    D.level_sch.assign(D.n_levels, 0);
    D.sch_entries[0] = D.sch_entries[1] = 0;
    for (int l = 0; l < D.n_levels; ++l) {
        int64_t acc = 0;
        for (int q = D.level_ptr[l]; q < D.level_ptr[l + 1]; ++q) {
            Front& F = D.fronts[D.level_fronts[q]];
            F.sch_off = acc;
            acc += (int64_t)F.u * F.u;
        }
        D.level_sch[l] = acc;
        D.sch_entries[l & 1] = std::max(D.sch_entries[l & 1], acc);
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
    // gather lists of the sweeps' extend-add
    D.asm_base.assign(nfr, 0);
    int64_t rows = 0;
    for (int64_t k = 0; k < nfr; ++k) {
        D.asm_base[k] = rows;
        rows += (int64_t)D.fronts[k].p + D.fronts[k].u;
    }
    D.asm_ptr.assign(rows + 1, 0);
    for (int64_t k = 0; k < nfr; ++k)
        for (int32_t q = D.child_ptr[k]; q < D.child_ptr[k + 1]; ++q) {
            const Front& C = D.fronts[D.child[q]];
            for (int32_t j = 0; j < C.u; ++j) D.asm_ptr[D.asm_base[k] + D.urel[C.u_off + j] + 1]++;
        }
    for (int64_t r = 0; r < rows; ++r) D.asm_ptr[r + 1] += D.asm_ptr[r];
    D.asm_src.assign(D.asm_ptr[rows], 0);
    {
        std::vector<int64_t> fill(D.asm_ptr.begin(), D.asm_ptr.end() - 1);
        for (int64_t k = 0; k < nfr; ++k)
            for (int32_t q = D.child_ptr[k]; q < D.child_ptr[k + 1]; ++q) {
                const Front& C = D.fronts[D.child[q]];
                for (int32_t j = 0; j < C.u; ++j)
                    D.asm_src[fill[D.asm_base[k] + D.urel[C.u_off + j]]++] = (int32_t)(C.upd_row + j);
            }
    }
}

}  // namespace mwi
