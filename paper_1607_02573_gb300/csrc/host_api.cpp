// C-ABI entry points that run the library's host logic without any device
// work, so that it can be checked without a GPU: the antenna map of the
// forward solve, the decomposition and its multifrontal structure, the
// assembly maps of A and of the B_i, and the coarse-space prolongation.  Each
// builds what it needs from the mesh arrays and copies it out; nothing is kept.
#include <algorithm>
#include <cstring>
#include <vector>

#include "common.h"
#include "model.h"

using namespace mwi;

namespace {

// the library's decomposition of a host mesh (the solver options' defaults for
// zero arguments), for the host-only entry points
void host_decomposition(const double* xyz, int64_t nv, const int32_t* tet, int64_t nt,
                               const int32_t* bface_tag, int32_t order, int32_t n_sub, int32_t overlap,
                               int32_t nd_leaf, Topology& T, Decomposition& D) {
    MWI_REQUIRE(xyz && tet && bface_tag, MWI_EINVAL, "null mesh array");
    mwi_solver_opts o;
    std::memset(&o, 0, sizeof(o));
    o.n_sub = n_sub;
    o.overlap = overlap;
    o.nd_leaf = nd_leaf;
    o = solver_defaults(&o);
    build_topology(T, xyz, nv, tet, nt, bface_tag, order);
    MWI_REQUIRE(o.n_sub <= T.nt, MWI_EINVAL, "more subdomains than tets");
    build_decomposition(T, nullptr, o.n_sub, o.overlap, o.nd_leaf, D);
}

}  // namespace

extern "C" {

mwi_status mwi_coarse_prolongation_host(const double* fxyz, int64_t fnv, const int32_t* ftet, int64_t fnt,
                                        const int32_t* fbface_tag, int32_t forder, const double* cxyz, int64_t cnv,
                                        const int32_t* ctet, int64_t cnt, const int32_t* cbface_tag, int64_t* n,
                                        int64_t* nc, int64_t* nnz, int64_t* p_rp, int32_t* p_col, double* p_val,
                                        int32_t* fkind, int64_t* fverts, int32_t* ckind, int64_t* cverts) {
    return guard([&] {
        MWI_REQUIRE(fxyz && ftet && fbface_tag && cxyz && ctet && cbface_tag, MWI_EINVAL, "null mesh array");
        Topology Tf, Tc;
        build_topology(Tf, fxyz, fnv, ftet, fnt, fbface_tag, forder);
        build_topology(Tc, cxyz, cnv, ctet, cnt, cbface_tag, 1);
        CoarseHost H;
        build_prolongation(Tf, Tc, H);
        if (n) *n = H.n;
        if (nc) *nc = H.nc;
        if (nnz) *nnz = (int64_t)H.P_col.size();
        if (p_rp) std::copy(H.P_rp.begin(), H.P_rp.end(), p_rp);
        if (p_col) std::copy(H.P_col.begin(), H.P_col.end(), p_col);
        if (p_val) std::copy(H.P_val.begin(), H.P_val.end(), p_val);
        if (fkind) std::copy(Tf.dof_kind.begin(), Tf.dof_kind.end(), fkind);
        if (fverts) std::copy(Tf.dof_verts.begin(), Tf.dof_verts.end(), fverts);
        if (ckind) std::copy(Tc.dof_kind.begin(), Tc.dof_kind.end(), ckind);
        if (cverts) std::copy(Tc.dof_verts.begin(), Tc.dof_verts.end(), cverts);
    });
}

mwi_status mwi_antenna_map_host(const double* xyz, int64_t nv, const int32_t* tet, int64_t nt,
                                const int32_t* bface_tag, int32_t order, const mwi_antenna* ants, int32_t n_ant,
                                int32_t* dof_out, double* sign_out, int64_t* ndof, int32_t* kind, int64_t* verts) {
    return guard([&] {
        MWI_REQUIRE(xyz && tet && bface_tag, MWI_EINVAL, "null mesh array");
        MWI_REQUIRE(n_ant >= 0 && (n_ant == 0 || ants), MWI_EINVAL, "null antennas");
        Topology T;
        build_topology(T, xyz, nv, tet, nt, bface_tag, order);
        std::vector<int32_t> dof;
        std::vector<double> sign;
        map_antennas(T, ants, n_ant, dof, sign);
        if (dof_out) std::copy(dof.begin(), dof.end(), dof_out);
        if (sign_out) std::copy(sign.begin(), sign.end(), sign_out);
        if (ndof) *ndof = T.ndof;
        if (kind) std::copy(T.dof_kind.begin(), T.dof_kind.end(), kind);
        if (verts) std::copy(T.dof_verts.begin(), T.dof_verts.end(), verts);
    });
}

mwi_status mwi_fronts_host(const double* xyz, int64_t nv, const int32_t* tet, int64_t nt, const int32_t* bface_tag,
                           int32_t order, int32_t n_sub, int32_t overlap, int32_t nd_leaf, int32_t* n_fronts,
                           int64_t* n_urows, int64_t* n_asm, int32_t* front_info, int64_t* u_off, int32_t* urows,
                           int32_t* urel, int64_t* asm_ptr, int32_t* asm_src) {
    return guard([&] {
        Topology T;
        Decomposition D;
        host_decomposition(xyz, nv, tet, nt, bface_tag, order, n_sub, overlap, nd_leaf, T, D);
        if (n_fronts) *n_fronts = (int32_t)D.fronts.size();
        if (n_urows) *n_urows = (int64_t)D.urows.size();
        for (size_t k = 0; k < D.fronts.size(); ++k) {
            const Front& F = D.fronts[k];
            if (front_info) {
                int32_t* q = front_info + 5 * k;
                q[0] = F.sub;
                q[1] = F.start;
                q[2] = F.p;
                q[3] = F.u;
                q[4] = F.parent;
            }
            if (u_off) u_off[k] = F.u_off;
        }
        if (urows) std::copy(D.urows.begin(), D.urows.end(), urows);
        if (n_asm) *n_asm = (int64_t)D.asm_src.size();
        if (urel) std::copy(D.urel.begin(), D.urel.end(), urel);
        if (asm_ptr) std::copy(D.asm_ptr.begin(), D.asm_ptr.end(), asm_ptr);
        if (asm_src) std::copy(D.asm_src.begin(), D.asm_src.end(), asm_src);
    });
}

mwi_status mwi_decomposition_host(const double* xyz, int64_t nv, const int32_t* tet, int64_t nt,
                                  const int32_t* bface_tag, int32_t order, int32_t n_sub, int32_t overlap,
                                  int32_t nd_leaf, int32_t* part, int64_t* sub_off, int32_t* loc2glob,
                                  double* dweight, int64_t* fu_off, int32_t* fu_verts, int32_t* fu_tet,
                                  int64_t* nloc, int64_t* nfu, int64_t* ndof, int32_t* kind, int64_t* verts,
                                  int64_t* factor_entries, int64_t* upd_rows) {
    return guard([&] {
        Topology T;
        Decomposition D;
        host_decomposition(xyz, nv, tet, nt, bface_tag, order, n_sub, overlap, nd_leaf, T, D);
        const FaceUses& F = D.B_faces;
        if (part) std::copy(D.part.begin(), D.part.end(), part);
        if (sub_off) std::copy(D.sub_off.begin(), D.sub_off.end(), sub_off);
        if (loc2glob) std::copy(D.loc2glob.begin(), D.loc2glob.end(), loc2glob);
        if (dweight) std::copy(D.dweight.begin(), D.dweight.end(), dweight);
        if (fu_off) std::copy(D.fu_off.begin(), D.fu_off.end(), fu_off);
        if (fu_verts)
            for (size_t k = 0; k < F.face.size(); ++k)
                for (int j = 0; j < 3; ++j) fu_verts[3 * k + j] = T.faces[3 * (int64_t)F.face[k] + j];
        if (fu_tet) std::copy(F.tet.begin(), F.tet.end(), fu_tet);
        if (nloc) *nloc = (int64_t)D.loc2glob.size();
        if (nfu) *nfu = (int64_t)F.face.size();
        if (ndof) *ndof = T.ndof;
        if (kind) std::copy(T.dof_kind.begin(), T.dof_kind.end(), kind);
        if (verts) std::copy(T.dof_verts.begin(), T.dof_verts.end(), verts);
        if (factor_entries) *factor_entries = D.factor_entries;
        if (upd_rows) *upd_rows = D.upd_rows;
    });
}

mwi_status mwi_slots_host(const double* xyz, int64_t nv, const int32_t* tet, int64_t nt, const int32_t* bface_tag,
                          int32_t order, int64_t* ndof, int64_t* nnz, int64_t* ncontrib, int64_t* nfu,
                          int64_t* row_ptr, int32_t* col, int64_t* slot_ptr, int64_t* contrib, int32_t* tet_dofs,
                          int32_t* fu_dofs, int32_t* fu_tet, int32_t* fu_verts, int32_t* kind, int64_t* verts) {
    return guard([&] {
        MWI_REQUIRE(xyz && tet && bface_tag, MWI_EINVAL, "null mesh array");
        Topology T;
        build_topology(T, xyz, nv, tet, nt, bface_tag, order);
        SlotMatrix A;
        FaceUses F;
        build_global_slots(T, A, F);
        if (ndof) *ndof = T.ndof;
        if (nnz) *nnz = (int64_t)A.col.size();
        if (ncontrib) *ncontrib = (int64_t)A.contrib.size();
        if (nfu) *nfu = (int64_t)F.face.size();
        if (row_ptr) std::copy(A.row_ptr.begin(), A.row_ptr.end(), row_ptr);
        if (col) std::copy(A.col.begin(), A.col.end(), col);
        if (slot_ptr) std::copy(A.slot_ptr.begin(), A.slot_ptr.end(), slot_ptr);
        if (contrib) std::copy(A.contrib.begin(), A.contrib.end(), contrib);
        if (tet_dofs) std::copy(T.tet_dofs.begin(), T.tet_dofs.end(), tet_dofs);
        for (size_t k = 0; k < F.face.size(); ++k) {
            const int64_t f = F.face[k];
            if (fu_dofs)
                for (int i = 0; i < T.nlf; ++i) fu_dofs[(int64_t)T.nlf * k + i] = T.face_dofs[(int64_t)T.nlf * f + i];
            if (fu_verts)
                for (int j = 0; j < 3; ++j) fu_verts[3 * k + j] = T.faces[3 * f + j];
        }
        if (fu_tet) std::copy(F.tet.begin(), F.tet.end(), fu_tet);
        if (kind) std::copy(T.dof_kind.begin(), T.dof_kind.end(), kind);
        if (verts) std::copy(T.dof_verts.begin(), T.dof_verts.end(), verts);
    });
}

mwi_status mwi_local_assembly_host(const double* xyz, int64_t nv, const int32_t* tet, int64_t nt,
                                   const int32_t* bface_tag, int32_t order, int32_t n_sub, int32_t overlap,
                                   int32_t nd_leaf, int64_t* nloc, int64_t* nslot, int64_t* ncontrib, int64_t* nfu,
                                   int64_t* namap, int32_t* n_fronts, int64_t* B_row_ptr, int32_t* B_col,
                                   int64_t* B_slot_ptr, int64_t* B_contrib, int32_t* fu_dofs,
                                   int64_t* amap_front_ptr, int64_t* amap_slot, int64_t* amap_pos) {
    return guard([&] {
        Topology T;
        Decomposition D;
        host_decomposition(xyz, nv, tet, nt, bface_tag, order, n_sub, overlap, nd_leaf, T, D);
        const SlotMatrix& B = D.B;
        if (nloc) *nloc = B.nrows;
        if (nslot) *nslot = (int64_t)B.col.size();
        if (ncontrib) *ncontrib = (int64_t)B.contrib.size();
        if (nfu) *nfu = (int64_t)D.B_faces.face.size();
        if (namap) *namap = (int64_t)D.amap_slot.size();
        if (n_fronts) *n_fronts = (int32_t)D.fronts.size();
        if (B_row_ptr) std::copy(B.row_ptr.begin(), B.row_ptr.end(), B_row_ptr);
        if (B_col) std::copy(B.col.begin(), B.col.end(), B_col);
        if (B_slot_ptr) std::copy(B.slot_ptr.begin(), B.slot_ptr.end(), B_slot_ptr);
        if (B_contrib) std::copy(B.contrib.begin(), B.contrib.end(), B_contrib);
        if (fu_dofs)
            for (size_t k = 0; k < D.B_faces.face.size(); ++k)
                for (int i = 0; i < T.nlf; ++i)
                    fu_dofs[(int64_t)T.nlf * k + i] = T.face_dofs[(int64_t)T.nlf * D.B_faces.face[k] + i];
        if (amap_front_ptr) std::copy(D.amap_front_ptr.begin(), D.amap_front_ptr.end(), amap_front_ptr);
        if (amap_slot) std::copy(D.amap_slot.begin(), D.amap_slot.end(), amap_slot);
        if (amap_pos) std::copy(D.amap_pos.begin(), D.amap_pos.end(), amap_pos);
    });
}

}  // extern "C"
