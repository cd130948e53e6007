// Mesh topology and DOF numbering (Section 2.1: Nedelec edge elements on a
// tetrahedral mesh; DOFs are attached to oriented edges, and for degree 2 also
// to faces).  Orientation: every tet's vertices are sorted by global id, so a
// local edge (i < j) runs from the lower to the higher global id and a face
// (a < b < c) has one canonical vertex order; no sign arrays are needed.
// DOFs on perfectly conducting faces are removed (Eq. eqmetal).  The internal
// DOF order follows the Morton (Z-order) code of the DOF's position so that
// neighbouring DOFs sit close in memory.
#include <algorithm>
#include <cmath>
#include <numeric>

#include "common.h"
#include "model.h"

namespace mwi {

static int local_edge_index(int a, int b) {
    for (int e = 0; e < 6; ++e)
        if ((kLocalEdges[e][0] == a && kLocalEdges[e][1] == b) ||
            (kLocalEdges[e][0] == b && kLocalEdges[e][1] == a))
            return e;
    return -1;
}

static uint64_t spread21(uint64_t x) {
    x &= 0x1fffff;
    x = (x | x << 32) & 0x1f00000000ffffULL;
    x = (x | x << 16) & 0x1f0000ff0000ffULL;
    x = (x | x << 8) & 0x100f00f00f00f00fULL;
    x = (x | x << 4) & 0x10c30c30c30c30c3ULL;
    x = (x | x << 2) & 0x1249249249249249ULL;
    return x;
}

static void build_csr(int64_t n, const std::vector<int32_t>& key, const std::vector<int32_t>& val,
                      std::vector<int32_t>& ptr, std::vector<int32_t>& out) {
    ptr.assign(n + 1, 0);
    for (int32_t k : key) ptr[k + 1]++;
    for (int64_t i = 0; i < n; ++i) ptr[i + 1] += ptr[i];
    out.resize(key.size());
    std::vector<int32_t> fill(ptr.begin(), ptr.end() - 1);
    for (size_t i = 0; i < key.size(); ++i) out[fill[key[i]]++] = val[i];
}

void build_topology(Topology& T, const double* xyz, int64_t nv, const int32_t* tet, int64_t nt,
                    const int32_t* bface_tag, int order) {
    MWI_REQUIRE(order == 1 || order == 2, MWI_EINVAL, "order must be 1 or 2");
    MWI_REQUIRE(nv >= 4 && nt >= 1, MWI_EINVAL, "mesh needs at least one tet");
    MWI_REQUIRE(nv < (int64_t)1 << 31 && nt < (int64_t)1 << 28, MWI_EINVAL, "mesh too large");
    T.order = order;
    T.nl = n_local(order);
    T.nlf = n_face_local(order);
    T.nv = nv;
    T.nt = nt;
    T.xyz.assign(xyz, xyz + nv * 3);

    T.centroid.resize(nt * 3);
    for (int64_t t = 0; t < nt; ++t)
        for (int d = 0; d < 3; ++d) {
            double s = xyz[3 * (int64_t)tet[4 * t] + d] + xyz[3 * (int64_t)tet[4 * t + 1] + d];
            s = s + xyz[3 * (int64_t)tet[4 * t + 2] + d];
            s = s + xyz[3 * (int64_t)tet[4 * t + 3] + d];
            T.centroid[3 * t + d] = s / 4.0;
        }
    // sorted tets and per-sorted-face tags
    T.tv.resize(nt * 4);
    std::vector<int8_t> ftag_tet(nt * 4);
    for (int64_t t = 0; t < nt; ++t) {
        int idx[4] = {0, 1, 2, 3};
        const int32_t* v = tet + 4 * t;
        for (int k = 0; k < 4; ++k) {
            MWI_REQUIRE(v[k] >= 0 && v[k] < nv, MWI_EINVAL, "tet vertex id out of range");
            int tg = bface_tag[4 * t + k];
            MWI_REQUIRE(tg >= 0 && tg <= 2, MWI_EINVAL, "bface_tag must be 0, 1 or 2");
        }
        std::sort(idx, idx + 4, [&](int a, int b) { return v[a] < v[b]; });
        for (int k = 0; k < 4; ++k) T.tv[4 * t + k] = v[idx[k]];
        for (int k = 0; k < 3; ++k)
            MWI_REQUIRE(T.tv[4 * t + k] != T.tv[4 * t + k + 1], MWI_EINVAL, "tet repeats a vertex");
        for (int f = 0; f < 4; ++f) ftag_tet[4 * t + f] = (int8_t)bface_tag[4 * t + idx[kOpposite[f]]];
        const double* p0 = xyz + 3 * (int64_t)T.tv[4 * t];
        double e[3][3];
        for (int k = 0; k < 3; ++k)
            for (int d = 0; d < 3; ++d) e[k][d] = xyz[3 * (int64_t)T.tv[4 * t + k + 1] + d] - p0[d];
        double det = e[0][0] * (e[1][1] * e[2][2] - e[1][2] * e[2][1]) -
                     e[0][1] * (e[1][0] * e[2][2] - e[1][2] * e[2][0]) +
                     e[0][2] * (e[1][0] * e[2][1] - e[1][1] * e[2][0]);
        MWI_REQUIRE(det != 0.0 && std::isfinite(det), MWI_EINVAL, "degenerate tetrahedron");
    }

    // edges
    {
        std::vector<std::pair<int64_t, int64_t>> ek(nt * 6);
        for (int64_t t = 0; t < nt; ++t)
            for (int e = 0; e < 6; ++e) {
                int64_t a = T.tv[4 * t + kLocalEdges[e][0]], b = T.tv[4 * t + kLocalEdges[e][1]];
                ek[6 * t + e] = {a * nv + b, 6 * t + e};
            }
        std::sort(ek.begin(), ek.end());
        T.tet_edges.resize(nt * 6);
        T.edges.clear();
        int64_t ne = -1, prev = -1;
        for (auto& kv : ek) {
            if (kv.first != prev) {
                ++ne;
                prev = kv.first;
                T.edges.push_back((int32_t)(kv.first / nv));
                T.edges.push_back((int32_t)(kv.first % nv));
            }
            T.tet_edges[kv.second] = (int32_t)ne;
        }
        T.ne = ne + 1;
    }
    // faces
    {
        std::vector<int64_t> idx(nt * 4);
        std::iota(idx.begin(), idx.end(), 0);
        auto fv = [&](int64_t i, int k) { return T.tv[4 * (i / 4) + kLocalFaces[i % 4][k]]; };
        std::sort(idx.begin(), idx.end(), [&](int64_t x, int64_t y) {
            for (int k = 0; k < 3; ++k) {
                int32_t a = fv(x, k), b = fv(y, k);
                if (a != b) return a < b;
            }
            return x < y;
        });
        T.tet_faces.resize(nt * 4);
        T.faces.clear();
        T.face_tag.clear();
        T.face_tets.clear();
        T.face_lf.clear();
        int64_t nf = -1;
        for (size_t q = 0; q < idx.size(); ++q) {
            int64_t i = idx[q];
            bool fresh = q == 0;
            if (!fresh) {
                int64_t j = idx[q - 1];
                fresh = fv(i, 0) != fv(j, 0) || fv(i, 1) != fv(j, 1) || fv(i, 2) != fv(j, 2);
            }
            if (fresh) {
                ++nf;
                for (int k = 0; k < 3; ++k) T.faces.push_back(fv(i, k));
                T.face_tag.push_back(ftag_tet[i]);
                T.face_tets.push_back((int32_t)(i / 4));
                T.face_tets.push_back(-1);
                T.face_lf.push_back((int8_t)(i % 4));
                T.face_lf.push_back(-1);
            } else {
                MWI_REQUIRE(T.face_tets[2 * nf + 1] < 0, MWI_EINVAL, "a face is shared by more than two tets");
                T.face_tets[2 * nf + 1] = (int32_t)(i / 4);
                T.face_lf[2 * nf + 1] = (int8_t)(i % 4);
                T.face_tag[nf] = std::max<int8_t>(T.face_tag[nf], ftag_tet[i]);
            }
            T.tet_faces[i] = (int32_t)nf;
        }
        T.nf = nf + 1;
    }

    // PEC entities
    T.pec_edge.assign(T.ne, 0);
    T.pec_face.assign(T.nf, 0);
    for (int64_t f = 0; f < T.nf; ++f) {
        if (T.face_tag[f] != TAG_PEC) continue;
        T.pec_face[f] = 1;
        int t = T.face_tets[2 * f], lf = T.face_lf[2 * f];
        for (int a = 0; a < 3; ++a)
            for (int b = a + 1; b < 3; ++b) {
                int e = local_edge_index(kLocalFaces[lf][a], kLocalFaces[lf][b]);
                T.pec_edge[T.tet_edges[6 * t + e]] = 1;
            }
    }

    // DOF candidates and Morton ordering
    struct Cand { uint64_t key; int kind; int64_t ent; };
    std::vector<Cand> cand;
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int64_t v = 0; v < nv; ++v)
        for (int d = 0; d < 3; ++d) {
            lo[d] = std::min(lo[d], xyz[3 * v + d]);
            hi[d] = std::max(hi[d], xyz[3 * v + d]);
        }
    double span = std::max({hi[0] - lo[0], hi[1] - lo[1], hi[2] - lo[2], 1e-300});
    auto morton = [&](const double* p) {
        uint64_t c[3];
        for (int d = 0; d < 3; ++d) {
            double s = (p[d] - lo[d]) / span;
            s = std::min(std::max(s, 0.0), 1.0);
            c[d] = (uint64_t)(s * 2097151.0);
        }
        return spread21(c[0]) | (spread21(c[1]) << 1) | (spread21(c[2]) << 2);
    };
    for (int64_t e = 0; e < T.ne; ++e) {
        if (T.pec_edge[e]) continue;
        double p[3];
        for (int d = 0; d < 3; ++d)
            p[d] = 0.5 * (xyz[3 * (int64_t)T.edges[2 * e] + d] + xyz[3 * (int64_t)T.edges[2 * e + 1] + d]);
        uint64_t k = morton(p);
        cand.push_back({k, KIND_WHITNEY, e});
        if (order == 2) cand.push_back({k, KIND_GRAD, e});
    }
    if (order == 2) {
        for (int64_t f = 0; f < T.nf; ++f) {
            if (T.pec_face[f]) continue;
            double p[3];
            for (int d = 0; d < 3; ++d) {
                p[d] = 0.0;
                for (int k = 0; k < 3; ++k) p[d] += xyz[3 * (int64_t)T.faces[3 * f + k] + d];
                p[d] /= 3.0;
            }
            uint64_t k = morton(p);
            cand.push_back({k, KIND_FACE_A, f});
            cand.push_back({k, KIND_FACE_B, f});
        }
    }
    std::sort(cand.begin(), cand.end(), [](const Cand& a, const Cand& b) {
        if (a.key != b.key) return a.key < b.key;
        if (a.ent != b.ent) return a.ent < b.ent;
        return a.kind < b.kind;
    });
    T.ndof = (int64_t)cand.size();
    MWI_REQUIRE(T.ndof > 0, MWI_EINVAL, "every DOF is on a PEC face");
    T.edge_dof.assign(T.ne, -1);
    std::vector<int32_t> grad_dof(order == 2 ? T.ne : 0, -1);
    std::vector<int32_t> facea_dof(order == 2 ? T.nf : 0, -1);
    T.dof_kind.resize(T.ndof);
    T.dof_verts.resize(T.ndof * 3);
    T.dof_pos.resize(T.ndof * 3);
    for (int64_t i = 0; i < T.ndof; ++i) {
        const Cand& c = cand[i];
        T.dof_kind[i] = c.kind;
        if (c.kind == KIND_WHITNEY || c.kind == KIND_GRAD) {
            if (c.kind == KIND_WHITNEY) T.edge_dof[c.ent] = (int32_t)i;
            else grad_dof[c.ent] = (int32_t)i;
            int64_t a = T.edges[2 * c.ent], b = T.edges[2 * c.ent + 1];
            T.dof_verts[3 * i] = a;
            T.dof_verts[3 * i + 1] = b;
            T.dof_verts[3 * i + 2] = -1;
            for (int d = 0; d < 3; ++d) T.dof_pos[3 * i + d] = 0.5 * (xyz[3 * a + d] + xyz[3 * b + d]);
        } else {
            if (c.kind == KIND_FACE_A) facea_dof[c.ent] = (int32_t)i;
            for (int k = 0; k < 3; ++k) T.dof_verts[3 * i + k] = T.faces[3 * c.ent + k];
            for (int d = 0; d < 3; ++d) {
                double s = 0;
                for (int k = 0; k < 3; ++k) s += xyz[3 * (int64_t)T.faces[3 * c.ent + k] + d];
                T.dof_pos[3 * i + d] = s / 3.0;
            }
        }
    }
    // the two DOFs of a face are adjacent in the ordering (same key, same entity)
    const int nl = T.nl;
    T.tet_dofs.assign(nt * nl, -1);
    for (int64_t t = 0; t < nt; ++t) {
        for (int e = 0; e < 6; ++e) {
            int32_t ed = T.tet_edges[6 * t + e];
            T.tet_dofs[nl * t + e] = T.edge_dof[ed];
            if (order == 2) T.tet_dofs[nl * t + 6 + e] = grad_dof[ed];
        }
        if (order == 2)
            for (int f = 0; f < 4; ++f) {
                int32_t fa = facea_dof[T.tet_faces[4 * t + f]];
                T.tet_dofs[nl * t + 12 + 2 * f] = fa;
                T.tet_dofs[nl * t + 13 + 2 * f] = fa >= 0 ? fa + 1 : -1;
            }
    }
    // face-local DOFs: W(ab, ac, bc) [, G(ab, ac, bc), Fa, Fb]
    const int nlf = T.nlf;
    T.face_dofs.assign(T.nf * nlf, -1);
    for (int64_t f = 0; f < T.nf; ++f) {
        int t = T.face_tets[2 * f], lf = T.face_lf[2 * f];
        const int* fl = kLocalFaces[lf];
        int le[3] = {local_edge_index(fl[0], fl[1]), local_edge_index(fl[0], fl[2]),
                     local_edge_index(fl[1], fl[2])};
        for (int k = 0; k < 3; ++k) {
            T.face_dofs[nlf * f + k] = T.tet_dofs[nl * t + le[k]];
            if (order == 2) T.face_dofs[nlf * f + 3 + k] = T.tet_dofs[nl * t + 6 + le[k]];
        }
        if (order == 2) {
            T.face_dofs[nlf * f + 6] = T.tet_dofs[nl * t + 12 + 2 * lf];
            T.face_dofs[nlf * f + 7] = T.tet_dofs[nl * t + 13 + 2 * lf];
        }
    }

    // adjacency lists
    {
        std::vector<int32_t> key, val;
        key.reserve(T.ne * 2);
        val.reserve(T.ne * 2);
        for (int64_t e = 0; e < T.ne; ++e) {
            key.push_back(T.edges[2 * e]); val.push_back((int32_t)e);
            key.push_back(T.edges[2 * e + 1]); val.push_back((int32_t)e);
        }
        build_csr(nv, key, val, T.v2e_ptr, T.v2e);
        for (int64_t v = 0; v < nv; ++v) std::sort(T.v2e.begin() + T.v2e_ptr[v], T.v2e.begin() + T.v2e_ptr[v + 1]);
    }
    {
        std::vector<int32_t> key(nt * 4), val(nt * 4);
        for (int64_t t = 0; t < nt; ++t)
            for (int k = 0; k < 4; ++k) { key[4 * t + k] = T.tv[4 * t + k]; val[4 * t + k] = (int32_t)t; }
        build_csr(nv, key, val, T.v2t_ptr, T.v2t);
    }
    {
        std::vector<int32_t> key, val;
        key.reserve(nt * nl);
        val.reserve(nt * nl);
        for (int64_t t = 0; t < nt; ++t)
            for (int i = 0; i < nl; ++i) {
                int32_t d = T.tet_dofs[nl * t + i];
                if (d >= 0) { key.push_back(d); val.push_back((int32_t)(t * nl + i)); }
            }
        build_csr(T.ndof, key, val, T.d2t_ptr, T.d2t);
    }
    build_vertex_grid(T.xyz, nv, T.vgrid);
}

}  // namespace mwi
