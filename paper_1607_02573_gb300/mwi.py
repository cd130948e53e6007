"""ctypes binding of libmwi.so: the C entry points under their C names, plus
two small handle classes that marshal NumPy / torch arrays.

Only argument marshalling happens here; every step of the computation runs
in the CUDA library.  Importing this module raises if the library has not
been built (``python -m paper_1607_02573_gb300.build``).
"""

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmwi.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with python -m paper_1607_02573_gb300.build")
_lib = C.CDLL(LIB_PATH)

MWI_OK, MWI_EINVAL, MWI_ENOMEM, MWI_ENOTCONV, MWI_ECUDA, MWI_ETIMEOUT, MWI_ESTATE, MWI_ESINGULAR = range(8)
STATUS_NAMES = ["MWI_OK", "MWI_EINVAL", "MWI_ENOMEM", "MWI_ENOTCONV", "MWI_ECUDA", "MWI_ETIMEOUT",
                "MWI_ESTATE", "MWI_ESINGULAR"]


class MwiError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 8 else status}: {msg}")
        self.status = status


class mwi_antenna(C.Structure):
    _fields_ = [("pos", C.c_double * 3), ("dir", C.c_double * 3), ("re_I", C.c_double), ("im_I", C.c_double)]


class mwi_solver_opts(C.Structure):
    _fields_ = [("rtol", C.c_double), ("max_iter", C.c_int32), ("restart", C.c_int32), ("n_sub", C.c_int32),
                ("overlap", C.c_int32), ("precision", C.c_int32), ("inner_iters", C.c_int32),
                ("inner_rtol", C.c_double), ("nd_leaf", C.c_int32), ("verbose", C.c_int32),
                ("part", C.POINTER(C.c_int32)), ("max_block", C.c_int32), ("sweep_engine", C.c_int32),
                ("block_krylov", C.c_int32), ("recycle", C.c_int32), ("factor_reuse", C.c_int32)]


class mwi_solve_info(C.Structure):
    _fields_ = [("iters_max", C.c_int32), ("inner_total", C.c_int32), ("n_converged", C.c_int32),
                ("n_perturbed", C.c_int32), ("resid_max", C.c_double), ("setup_ms", C.c_double),
                ("solve_ms", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_vp = C.c_void_p
_dp = C.POINTER(C.c_double)
_i32p = C.POINTER(C.c_int32)
_i64p = C.POINTER(C.c_int64)

_SIGS = {
    "mwi_mesh_create": [_dp, C.c_int64, _i32p, C.c_int64, _i32p, C.c_int32, C.POINTER(_vp)],
    "mwi_mesh_ndof": [_vp, _i64p],
    "mwi_mesh_dof_keys": [_vp, _i32p, _i64p],
    "mwi_mesh_destroy": [_vp],
    "mwi_assemble": [_vp, _dp, C.c_double, C.POINTER(mwi_solver_opts), _vp, C.POINTER(_vp)],
    "mwi_assemble_device": [_vp, _vp, C.c_double, C.POINTER(mwi_solver_opts), _vp, C.POINTER(_vp)],
    "mwi_update_eps": [_vp, _dp],
    "mwi_update_eps_device": [_vp, _vp],
    "mwi_forward_solve": [_vp, C.POINTER(mwi_antenna), C.c_int32, C.POINTER(mwi_antenna), C.c_int32, _dp,
                          C.POINTER(mwi_solve_info)],
    "mwi_misfit_and_gradient": [_vp, _dp, _dp, _dp, _dp, C.POINTER(mwi_solve_info)],
    "mwi_misfit_and_gradient_device": [_vp, _vp, _vp, _dp, _vp, C.POINTER(mwi_solve_info)],
    "mwi_fields_device": [_vp, C.c_int32, C.POINTER(_vp), _i64p, _i64p],
    "mwi_copy_fields": [_vp, C.c_int32, _dp],
    "mwi_problem_destroy": [_vp],
    "mwi_spmm_device": [_vp, _vp, _vp, C.c_int32],
    "mwi_oras_apply_device": [_vp, _vp, _vp, C.c_int32],
    "mwi_oras_apply_device_noalloc": [_vp, _vp, _vp, C.c_int32],
    "mwi_matrix_csr": [_vp, _i64p, _i64p, _i32p, _dp],
    "mwi_decomposition": [_vp, _i32p, _i64p],
    "mwi_factor_stats": [_vp, _i64p, _i64p, _i64p, _dp],
    "mwi_problem_device_bytes": [_vp, _i64p],
    "mwi_problem_estimate_bytes": [_vp, C.POINTER(mwi_solver_opts), C.c_int32, _i64p],
    "mwi_recycle_from": [_vp, _vp],
    "mwi_sweep_levels": [_vp, C.c_int32, _i32p, _i64p, _i64p, _i64p, _i64p, _i64p],
    "mwi_oras_traffic": [_vp, C.c_int32, _dp],
    "mwi_update_kappa_device": [_vp, _vp],
    "mwi_misfit_and_gradient_kappa_device": [_vp, _vp, _vp, C.c_double, _dp, _dp, _vp, C.POINTER(mwi_solve_info)],
    "mwi_normalised_weights": [_dp, C.c_int64, _dp],
    "mwi_kernel_times": [_vp, _dp, _i64p, C.c_int32],
    "mwi_misfit": [_vp, _dp, _dp, _dp],
    "mwi_set_coarse_space": [_vp, _vp],
    "mwi_coarse_info": [_vp, _i64p, _i64p, _i64p, _dp, _i32p],
    "mwi_coarse_operator": [_vp, _i64p, _i32p, _dp, _i64p, _i32p, _dp],
    "mwi_coarse_prolongation_host": [_dp, C.c_int64, _i32p, C.c_int64, _i32p, C.c_int32, _dp, C.c_int64, _i32p,
                                     C.c_int64, _i32p, _i64p, _i64p, _i64p, _i64p, _i32p, _dp, _i32p, _i64p, _i32p,
                                     _i64p],
    "mwi_antenna_map_host": [_dp, C.c_int64, _i32p, C.c_int64, _i32p, C.c_int32, C.POINTER(mwi_antenna), C.c_int32,
                             _i32p, _dp, _i64p, _i32p, _i64p],
    "mwi_decomposition_host": [_dp, C.c_int64, _i32p, C.c_int64, _i32p, C.c_int32, C.c_int32, C.c_int32, C.c_int32,
                               _i32p, _i64p, _i32p, _dp, _i64p, _i32p, _i32p, _i64p, _i64p, _i64p, _i32p, _i64p,
                               _i64p, _i64p],
    "mwi_fronts_host": [_dp, C.c_int64, _i32p, C.c_int64, _i32p, C.c_int32, C.c_int32, C.c_int32, C.c_int32, _i32p,
                        _i64p, _i64p, _i32p, _i64p, _i32p, _i32p, _i64p, _i32p],
    "mwi_slots_host": [_dp, C.c_int64, _i32p, C.c_int64, _i32p, C.c_int32, _i64p, _i64p, _i64p, _i64p, _i64p, _i32p,
                       _i64p, _i64p, _i32p, _i32p, _i32p, _i32p, _i32p, _i64p],
    "mwi_local_assembly_host": [_dp, C.c_int64, _i32p, C.c_int64, _i32p, C.c_int32, C.c_int32, C.c_int32, C.c_int32,
                                _i64p, _i64p, _i64p, _i64p, _i64p, _i32p, _i64p, _i32p, _i64p, _i64p, _i32p, _i64p,
                                _i64p, _i64p],
}
EXPORTED = sorted(list(_SIGS) + ["mwi_last_error", "mwi_launch_count", "mwi_device_alloc_count"])

for _name, _args in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = C.c_int
    globals()[_name] = _f
_lib.mwi_last_error.argtypes = []
_lib.mwi_last_error.restype = C.c_char_p
mwi_last_error = _lib.mwi_last_error
_lib.mwi_launch_count.argtypes = []
_lib.mwi_launch_count.restype = C.c_int64
mwi_launch_count = _lib.mwi_launch_count
_lib.mwi_device_alloc_count.argtypes = []
_lib.mwi_device_alloc_count.restype = C.c_int64
mwi_device_alloc_count = _lib.mwi_device_alloc_count


def check(status, allow=()):
    if status != MWI_OK and status not in allow:
        raise MwiError(status, (mwi_last_error() or b"").decode())
    return status


def coarse_prolongation_host(fine, coarse, fine_order=1):
    """The prolongation of the two-level ORAS between two meshes (objects with
    xyz, tet, bface_tag, nv), computed on the host (mwi_coarse_prolongation_host):
    (P as scipy CSR in the library's DOF numbering, (fine kind, fine verts),
    (coarse kind, coarse verts))."""
    import scipy.sparse as sp

    def arrs(m):
        return (np.ascontiguousarray(m.xyz, dtype=np.float64), np.ascontiguousarray(m.tet, dtype=np.int32),
                np.ascontiguousarray(m.bface_tag, dtype=np.int32))

    fx, ft, fb = arrs(fine)
    cx, ct, cb = arrs(coarse)
    n, nc, nnz = C.c_int64(), C.c_int64(), C.c_int64()
    head = [_ptr(fx, C.c_double), fx.shape[0], _ptr(ft, C.c_int32), ft.shape[0], _ptr(fb, C.c_int32), fine_order,
            _ptr(cx, C.c_double), cx.shape[0], _ptr(ct, C.c_int32), ct.shape[0], _ptr(cb, C.c_int32)]
    check(mwi_coarse_prolongation_host(*head, C.byref(n), C.byref(nc), C.byref(nnz), None, None, None, None, None,
                                       None, None))
    rp = np.empty(n.value + 1, dtype=np.int64)
    col = np.empty(nnz.value, dtype=np.int32)
    val = np.empty(nnz.value, dtype=np.float64)
    fk = np.empty(n.value, dtype=np.int32)
    fv = np.empty((n.value, 3), dtype=np.int64)
    ck = np.empty(nc.value, dtype=np.int32)
    cv = np.empty((nc.value, 3), dtype=np.int64)
    check(mwi_coarse_prolongation_host(*head, C.byref(n), C.byref(nc), C.byref(nnz), _ptr(rp, C.c_int64),
                                       _ptr(col, C.c_int32), _ptr(val, C.c_double), _ptr(fk, C.c_int32),
                                       _ptr(fv, C.c_int64), _ptr(ck, C.c_int32), _ptr(cv, C.c_int64)))
    return sp.csr_matrix((val, col, rp), shape=(n.value, nc.value)), (fk, fv), (ck, cv)


def antenna_map_host(mesh, antennas, order=1):
    """The antenna -> (edge DOF, sign) map of the forward solve for a mesh
    (xyz, tet, bface_tag), computed on the host (mwi_antenna_map_host):
    (dof [n], sign [n], (kind, verts) DOF keys of the library's numbering)."""
    x = np.ascontiguousarray(mesh.xyz, dtype=np.float64)
    t = np.ascontiguousarray(mesh.tet, dtype=np.int32)
    b = np.ascontiguousarray(mesh.bface_tag, dtype=np.int32)
    a = _antennas(antennas)
    n = len(a)
    head = [_ptr(x, C.c_double), x.shape[0], _ptr(t, C.c_int32), t.shape[0], _ptr(b, C.c_int32), order, a, n]
    ndof = C.c_int64()
    check(mwi_antenna_map_host(*head, None, None, C.byref(ndof), None, None))
    dof = np.empty(n, dtype=np.int32)
    sign = np.empty(n, dtype=np.float64)
    kind = np.empty(ndof.value, dtype=np.int32)
    verts = np.empty((ndof.value, 3), dtype=np.int64)
    check(mwi_antenna_map_host(*head, _ptr(dof, C.c_int32), _ptr(sign, C.c_double), C.byref(ndof),
                               _ptr(kind, C.c_int32), _ptr(verts, C.c_int64)))
    return dof, sign, (kind, verts)


def decomposition_host(mesh, n_sub, overlap=0, nd_leaf=0, order=1):
    """The ORAS decomposition of a mesh (xyz, tet, bface_tag), computed on the
    host (mwi_decomposition_host); overlap and nd_leaf as in the solver options
    (0: defaults).  Returns a dict: part [nt], sub_off [n_sub+1], loc2glob,
    dweight [nloc], fu_off [n_sub+1], fu_verts [nfu, 3], fu_tet [nfu], kind,
    verts (DOF keys), factor_entries, upd_rows."""
    x = np.ascontiguousarray(mesh.xyz, dtype=np.float64)
    t = np.ascontiguousarray(mesh.tet, dtype=np.int32)
    b = np.ascontiguousarray(mesh.bface_tag, dtype=np.int32)
    head = [_ptr(x, C.c_double), x.shape[0], _ptr(t, C.c_int32), t.shape[0], _ptr(b, C.c_int32), order, n_sub,
            overlap, nd_leaf]
    nloc, nfu, ndof, fe, ur = C.c_int64(), C.c_int64(), C.c_int64(), C.c_int64(), C.c_int64()
    sizes = [C.byref(nloc), C.byref(nfu), C.byref(ndof)]
    check(mwi_decomposition_host(*head, *([None] * 7), *sizes, None, None, None, None))
    ns = int(n_sub) if n_sub > 0 else 64
    out = dict(part=np.empty(t.shape[0], dtype=np.int32), sub_off=np.empty(ns + 1, dtype=np.int64),
               loc2glob=np.empty(nloc.value, dtype=np.int32), dweight=np.empty(nloc.value, dtype=np.float64),
               fu_off=np.empty(ns + 1, dtype=np.int64), fu_verts=np.empty((nfu.value, 3), dtype=np.int32),
               fu_tet=np.empty(nfu.value, dtype=np.int32), kind=np.empty(ndof.value, dtype=np.int32),
               verts=np.empty((ndof.value, 3), dtype=np.int64))
    check(mwi_decomposition_host(*head, _ptr(out["part"], C.c_int32), _ptr(out["sub_off"], C.c_int64),
                                 _ptr(out["loc2glob"], C.c_int32), _ptr(out["dweight"], C.c_double),
                                 _ptr(out["fu_off"], C.c_int64), _ptr(out["fu_verts"], C.c_int32),
                                 _ptr(out["fu_tet"], C.c_int32), *sizes, _ptr(out["kind"], C.c_int32),
                                 _ptr(out["verts"], C.c_int64), C.byref(fe), C.byref(ur)))
    out["factor_entries"], out["upd_rows"] = fe.value, ur.value
    return out


def fronts_host(mesh, n_sub, overlap=0, nd_leaf=0, order=1):
    """The multifrontal structure of the decomposition (mwi_fronts_host) as a
    dict: info [n_fronts, 5] = (sub, start, p, u, parent), u_off [n_fronts],
    urows, urel, asm_ptr, asm_src."""
    x = np.ascontiguousarray(mesh.xyz, dtype=np.float64)
    t = np.ascontiguousarray(mesh.tet, dtype=np.int32)
    b = np.ascontiguousarray(mesh.bface_tag, dtype=np.int32)
    head = [_ptr(x, C.c_double), x.shape[0], _ptr(t, C.c_int32), t.shape[0], _ptr(b, C.c_int32), order, n_sub,
            overlap, nd_leaf]
    nf, nu, na = C.c_int32(), C.c_int64(), C.c_int64()
    sizes = [C.byref(nf), C.byref(nu), C.byref(na)]
    check(mwi_fronts_host(*head, *sizes, *([None] * 6)))
    out = dict(info=np.empty((nf.value, 5), dtype=np.int32), u_off=np.empty(nf.value, dtype=np.int64),
               urows=np.empty(nu.value, dtype=np.int32), urel=np.empty(nu.value, dtype=np.int32))
    check(mwi_fronts_host(*head, *sizes, _ptr(out["info"], C.c_int32), _ptr(out["u_off"], C.c_int64),
                          _ptr(out["urows"], C.c_int32), _ptr(out["urel"], C.c_int32), None, None))
    nrows = int((out["info"][:, 2].astype(np.int64) + out["info"][:, 3]).sum())
    out["asm_ptr"] = np.empty(nrows + 1, dtype=np.int64)
    out["asm_src"] = np.empty(na.value, dtype=np.int32)
    check(mwi_fronts_host(*head, *sizes, None, None, None, None, _ptr(out["asm_ptr"], C.c_int64),
                          _ptr(out["asm_src"], C.c_int32)))
    return out


def slots_host(mesh, order=1):
    """The assembly map of A (mwi_slots_host) as a dict: row_ptr, col,
    slot_ptr, contrib, tet_dofs [nt, nl], fu_dofs [nfu, nlf], fu_tet, fu_verts
    [nfu, 3], kind, verts."""
    x = np.ascontiguousarray(mesh.xyz, dtype=np.float64)
    t = np.ascontiguousarray(mesh.tet, dtype=np.int32)
    b = np.ascontiguousarray(mesh.bface_tag, dtype=np.int32)
    head = [_ptr(x, C.c_double), x.shape[0], _ptr(t, C.c_int32), t.shape[0], _ptr(b, C.c_int32), order]
    n, nnz, nc, nfu = C.c_int64(), C.c_int64(), C.c_int64(), C.c_int64()
    sizes = [C.byref(n), C.byref(nnz), C.byref(nc), C.byref(nfu)]
    check(mwi_slots_host(*head, *sizes, *([None] * 10)))
    nl, nlf = (6, 3) if order == 1 else (20, 8)
    out = dict(row_ptr=np.empty(n.value + 1, dtype=np.int64), col=np.empty(nnz.value, dtype=np.int32),
               slot_ptr=np.empty(nnz.value + 1, dtype=np.int64), contrib=np.empty(nc.value, dtype=np.int64),
               tet_dofs=np.empty((t.shape[0], nl), dtype=np.int32), fu_dofs=np.empty((nfu.value, nlf), dtype=np.int32),
               fu_tet=np.empty(nfu.value, dtype=np.int32), fu_verts=np.empty((nfu.value, 3), dtype=np.int32),
               kind=np.empty(n.value, dtype=np.int32), verts=np.empty((n.value, 3), dtype=np.int64))
    check(mwi_slots_host(*head, *sizes, _ptr(out["row_ptr"], C.c_int64), _ptr(out["col"], C.c_int32),
                         _ptr(out["slot_ptr"], C.c_int64), _ptr(out["contrib"], C.c_int64),
                         _ptr(out["tet_dofs"], C.c_int32), _ptr(out["fu_dofs"], C.c_int32),
                         _ptr(out["fu_tet"], C.c_int32), _ptr(out["fu_verts"], C.c_int32),
                         _ptr(out["kind"], C.c_int32), _ptr(out["verts"], C.c_int64)))
    return out


def local_assembly_host(mesh, n_sub, overlap=0, nd_leaf=0, order=1):
    """The local operators' assembly maps (mwi_local_assembly_host) as a dict:
    B_row_ptr, B_col, B_slot_ptr, B_contrib, fu_dofs [nfu, nlf],
    amap_front_ptr, amap_slot, amap_pos."""
    x = np.ascontiguousarray(mesh.xyz, dtype=np.float64)
    t = np.ascontiguousarray(mesh.tet, dtype=np.int32)
    b = np.ascontiguousarray(mesh.bface_tag, dtype=np.int32)
    head = [_ptr(x, C.c_double), x.shape[0], _ptr(t, C.c_int32), t.shape[0], _ptr(b, C.c_int32), order, n_sub,
            overlap, nd_leaf]
    nloc, nslot, nc, nfu, nam = (C.c_int64() for _ in range(5))
    nf = C.c_int32()
    sizes = [C.byref(nloc), C.byref(nslot), C.byref(nc), C.byref(nfu), C.byref(nam), C.byref(nf)]
    check(mwi_local_assembly_host(*head, *sizes, *([None] * 8)))
    nlf = 3 if order == 1 else 8
    out = dict(B_row_ptr=np.empty(nloc.value + 1, dtype=np.int64), B_col=np.empty(nslot.value, dtype=np.int32),
               B_slot_ptr=np.empty(nslot.value + 1, dtype=np.int64), B_contrib=np.empty(nc.value, dtype=np.int64),
               fu_dofs=np.empty((nfu.value, nlf), dtype=np.int32),
               amap_front_ptr=np.empty(nf.value + 1, dtype=np.int64), amap_slot=np.empty(nam.value, dtype=np.int64),
               amap_pos=np.empty(nam.value, dtype=np.int64))
    check(mwi_local_assembly_host(*head, *sizes, *(_ptr(out[k], C.c_int32 if out[k].dtype == np.int32 else C.c_int64)
                                                   for k in ("B_row_ptr", "B_col", "B_slot_ptr", "B_contrib",
                                                             "fu_dofs", "amap_front_ptr", "amap_slot",
                                                             "amap_pos"))))
    return out


def normalised_weights(S_empty):
    """w_ij = 1 / |S_empty_ij|^2 (Eq. defJ2), computed by the library."""
    S = np.ascontiguousarray(S_empty, dtype=np.complex128)
    w = np.empty(S.shape, dtype=np.float64)
    check(mwi_normalised_weights(_ptr(S.view(np.float64), C.c_double), S.size, _ptr(w, C.c_double)))
    return w


def _ptr(a, ctype):
    return a.ctypes.data_as(C.POINTER(ctype))


def _antennas(arr):
    arr = np.asarray(arr, dtype=np.float64).reshape(-1, 8)
    out = (mwi_antenna * arr.shape[0])()
    for i, row in enumerate(arr):
        out[i].pos[:] = row[0:3]
        out[i].dir[:] = row[3:6]
        out[i].re_I = row[6]
        out[i].im_I = row[7]
    return out


def make_opts(**kw):
    o = mwi_solver_opts()
    part = kw.pop("part", None)
    names = {f for f, _ in mwi_solver_opts._fields_}
    for k, v in kw.items():
        if k not in names:
            raise TypeError(f"unknown solver option {k!r}")
        setattr(o, k, v)
    keep = None
    if part is not None:
        keep = np.ascontiguousarray(part, dtype=np.int32)
        o.part = _ptr(keep, C.c_int32)
    return o, keep


class Mesh:
    """Owns an mwi_mesh_t."""

    def __init__(self, xyz, tet, bface_tag, order=1):
        self.xyz = np.ascontiguousarray(xyz, dtype=np.float64)
        self.tet = np.ascontiguousarray(tet, dtype=np.int32)
        tag = np.ascontiguousarray(bface_tag, dtype=np.int32)
        self.nt = self.tet.shape[0]
        self.nv = self.xyz.shape[0]
        self.order = order
        h = _vp()
        check(mwi_mesh_create(_ptr(self.xyz, C.c_double), self.xyz.shape[0], _ptr(self.tet, C.c_int32), self.nt,
                              _ptr(tag, C.c_int32), order, C.byref(h)))
        self.h = h
        n = C.c_int64()
        check(mwi_mesh_ndof(h, C.byref(n)))
        self.ndof = n.value

    def estimate_bytes(self, n_rhs, **opts):
        """Upper estimate of the device bytes of a problem on this mesh (mwi_problem_estimate_bytes)."""
        o, keep = make_opts(**opts)
        b = C.c_int64()
        check(mwi_problem_estimate_bytes(self.h, C.byref(o), int(n_rhs), C.byref(b)))
        return b.value

    def dof_keys(self):
        kind = np.empty(self.ndof, dtype=np.int32)
        verts = np.empty((self.ndof, 3), dtype=np.int64)
        check(mwi_mesh_dof_keys(self.h, _ptr(kind, C.c_int32), _ptr(verts, C.c_int64)))
        return kind, verts

    def close(self):
        if self.h:
            check(mwi_mesh_destroy(self.h))
            self.h = None

    def __del__(self):
        try:
            if self.h:
                mwi_mesh_destroy(self.h)
        except Exception:
            pass


class Problem:
    """Owns an mwi_problem_t (assembled operator, ORAS factors, resident fields).

    Keyword options are the fields of mwi_solver_opts (include/mwi.h): rtol,
    max_iter, restart, n_sub, overlap, precision (0 FP64, 1 mixed, 2 nested),
    inner_iters, inner_rtol, nd_leaf, verbose, part, max_block, sweep_engine,
    block_krylov, recycle, factor_reuse; an unknown name raises TypeError."""

    def __init__(self, mesh, eps, freq, stream=None, **opts):
        import torch

        self.mesh = mesh
        self.freq = freq
        self.opts, self._part = make_opts(**opts)
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        h = _vp()
        if isinstance(eps, torch.Tensor):
            e = eps.to(torch.complex128).contiguous()
            check(mwi_assemble_device(mesh.h, _vp(e.data_ptr()), freq, C.byref(self.opts),
                                      _vp(stream.cuda_stream), C.byref(h)))
        else:
            e = np.ascontiguousarray(eps, dtype=np.complex128)
            check(mwi_assemble(mesh.h, _ptr(e.view(np.float64), C.c_double), freq, C.byref(self.opts),
                               _vp(stream.cuda_stream), C.byref(h)))
        self.h = h
        self.info = mwi_solve_info()

    def update_eps(self, eps):
        import torch
        if isinstance(eps, torch.Tensor):
            e = eps.to(torch.complex128).contiguous()
            check(mwi_update_eps_device(self.h, _vp(e.data_ptr())))
        else:
            e = np.ascontiguousarray(eps, dtype=np.complex128)
            check(mwi_update_eps(self.h, _ptr(e.view(np.float64), C.c_double)))

    def forward_solve(self, tx, rx, allow_notconv=False):
        t = _antennas(tx)
        r = _antennas(rx)
        S = np.empty((len(t), len(r)), dtype=np.complex128)  # column-major [n_rx, n_tx] == row-major [n_tx, n_rx]
        info = mwi_solve_info()
        st = mwi_forward_solve(self.h, t, len(t), r, len(r), _ptr(S.view(np.float64), C.c_double), C.byref(info))
        check(st, allow=(MWI_ENOTCONV,) if allow_notconv else ())
        self.info = info
        return S.T.copy()

    def misfit_and_gradient(self, S_meas, w=None, allow_notconv=False):
        S_meas = np.asfortranarray(S_meas, dtype=np.complex128)
        Sm = np.ascontiguousarray(S_meas.T)  # column-major storage of [n_rx, n_tx]
        wp = None
        if w is not None:
            wc = np.ascontiguousarray(np.asarray(w, dtype=np.float64).T)
            wp = _ptr(wc, C.c_double)
        J = C.c_double()
        grad = np.empty(self.mesh.nt, dtype=np.complex128)
        info = mwi_solve_info()
        st = mwi_misfit_and_gradient(self.h, _ptr(Sm.view(np.float64), C.c_double), wp, C.byref(J),
                                     _ptr(grad.view(np.float64), C.c_double), C.byref(info))
        check(st, allow=(MWI_ENOTCONV,) if allow_notconv else ())
        self.info = info
        return J.value, grad

    def misfit_and_gradient_device(self, S_meas, w=None, allow_notconv=False):
        """J and the per-tet gradient as a device tensor [nt] (measurements and weights from host arrays)."""
        import torch
        dev = torch.device("cuda", torch.cuda.current_device())
        Sm = torch.from_numpy(np.ascontiguousarray(np.asarray(S_meas, dtype=np.complex128).T)).to(dev)
        wd = None
        if w is not None:
            wd = torch.from_numpy(np.ascontiguousarray(np.asarray(w, dtype=np.float64).T)).to(dev)
        grad = torch.empty(self.mesh.nt, dtype=torch.complex128, device=dev)
        J = C.c_double()
        info = mwi_solve_info()
        st = mwi_misfit_and_gradient_device(self.h, _vp(Sm.data_ptr()), _vp(wd.data_ptr()) if wd is not None else None,
                                            C.byref(J), _vp(grad.data_ptr()), C.byref(info))
        check(st, allow=(MWI_ENOTCONV,) if allow_notconv else ())
        self.info = info
        return J.value, grad

    def update_kappa(self, kappa):
        """Reassemble (and refactor) for the nodal parameter kappa (device tensor [nv])."""
        import torch
        k = kappa.to(torch.complex128).contiguous()
        check(mwi_update_kappa_device(self.h, _vp(k.data_ptr())))

    def misfit_and_gradient_kappa(self, S_meas, w=None, alpha=0.0, allow_notconv=False):
        """J, R and the per-vertex gradient of J + R (device tensor [nv]) for the
        nodal parameter of the last update_kappa; S_meas, w host arrays [n_rx, n_tx]."""
        import torch
        dev = torch.device("cuda", torch.cuda.current_device())
        Sm = torch.from_numpy(np.ascontiguousarray(np.asarray(S_meas, dtype=np.complex128).T)).to(dev)
        wd = None
        if w is not None:
            wd = torch.from_numpy(np.ascontiguousarray(np.asarray(w, dtype=np.float64).T)).to(dev)
        grad = torch.empty(self.mesh.nv, dtype=torch.complex128, device=dev)
        J, R = C.c_double(), C.c_double()
        info = mwi_solve_info()
        st = mwi_misfit_and_gradient_kappa_device(self.h, _vp(Sm.data_ptr()),
                                                  _vp(wd.data_ptr()) if wd is not None else None, float(alpha),
                                                  C.byref(J), C.byref(R), _vp(grad.data_ptr()), C.byref(info))
        check(st, allow=(MWI_ENOTCONV,) if allow_notconv else ())
        self.info = info
        return J.value, R.value, grad

    def sweep_levels(self):
        """Per tree level (deepest first): fronts, panel entries, update rows and
        the 128-row tiles of the forward and backward tensor-core products."""
        n = C.c_int32()
        arr = [np.zeros(64, dtype=np.int64) for _ in range(5)]
        check(mwi_sweep_levels(self.h, 64, C.byref(n), *[_ptr(a, C.c_int64) for a in arr]))
        names = ["fronts", "panel_entries", "update_rows", "tiles_fwd", "tiles_bwd"]
        return {k: a[:n.value].tolist() for k, a in zip(names, arr)}

    def recycle_from(self, other):
        """Take the resident solutions of another problem on the same mesh (a
        nearby frequency) as this problem's recycled space (mwi_recycle_from)."""
        check(mwi_recycle_from(self.h, other.h))

    def set_coarse_space(self, coarse_mesh):
        """Two-level ORAS with the lowest-order Whitney space of coarse_mesh
        (a Mesh of order 1) as coarse space; None removes it."""
        check(mwi_set_coarse_space(self.h, coarse_mesh.h if coarse_mesh is not None else None))

    def coarse_info(self):
        nc, nnz_p, nnz_ac = C.c_int64(), C.c_int64(), C.c_int64()
        ms = C.c_double()
        npert = C.c_int32()
        check(mwi_coarse_info(self.h, C.byref(nc), C.byref(nnz_p), C.byref(nnz_ac), C.byref(ms), C.byref(npert)))
        return dict(n_coarse=nc.value, nnz_p=nnz_p.value, nnz_ac=nnz_ac.value, setup_ms=ms.value,
                    n_perturbed=npert.value)

    def coarse_operator(self):
        """(P, A_c) as scipy CSR matrices (library DOF order on both meshes)."""
        import scipy.sparse as sp
        info = self.coarse_info()
        n, nc = self.mesh.ndof, info["n_coarse"]
        p_rp = np.empty(n + 1, dtype=np.int64)
        p_col = np.empty(info["nnz_p"], dtype=np.int32)
        p_val = np.empty(info["nnz_p"], dtype=np.float64)
        a_rp = np.empty(nc + 1, dtype=np.int64)
        a_col = np.empty(info["nnz_ac"], dtype=np.int32)
        a_val = np.empty(info["nnz_ac"], dtype=np.complex128)
        check(mwi_coarse_operator(self.h, _ptr(p_rp, C.c_int64), _ptr(p_col, C.c_int32), _ptr(p_val, C.c_double),
                                  _ptr(a_rp, C.c_int64), _ptr(a_col, C.c_int32),
                                  _ptr(a_val.view(np.float64), C.c_double)))
        return (sp.csr_matrix((p_val, p_col, p_rp), shape=(n, nc)),
                sp.csr_matrix((a_val, a_col, a_rp), shape=(nc, nc)))

    def fields(self, which=0):
        """Borrowed device pointer and shape (n, m) of the resident fields."""
        p = _vp()
        n = C.c_int64()
        m = C.c_int64()
        check(mwi_fields_device(self.h, which, C.byref(p), C.byref(n), C.byref(m)))
        return p.value, n.value, m.value

    def fields_host(self, which=0):
        """Copy of the resident fields [n, m] (internal DOF order)."""
        _, n, m = self.fields(which)
        out = np.empty((n, m), dtype=np.complex128)
        check(mwi_copy_fields(self.h, which, _ptr(out.view(np.float64), C.c_double)))
        return out

    def spmm(self, x):
        import torch
        y = torch.empty_like(x)
        check(mwi_spmm_device(self.h, _vp(x.data_ptr()), _vp(y.data_ptr()), x.shape[1]))
        return y

    def oras_apply(self, x):
        import torch
        y = torch.empty_like(x)
        check(mwi_oras_apply_device(self.h, _vp(x.data_ptr()), _vp(y.data_ptr()), x.shape[1]))
        return y

    def matrix_csr(self):
        nnz = C.c_int64()
        check(mwi_matrix_csr(self.h, C.byref(nnz), None, None, None))
        rp = np.empty(self.mesh.ndof + 1, dtype=np.int64)
        col = np.empty(nnz.value, dtype=np.int32)
        val = np.empty(nnz.value, dtype=np.complex128)
        check(mwi_matrix_csr(self.h, C.byref(nnz), _ptr(rp, C.c_int64), _ptr(col, C.c_int32),
                             _ptr(val.view(np.float64), C.c_double)))
        return rp, col, val

    def decomposition(self, n_sub):
        part = np.empty(self.mesh.nt, dtype=np.int32)
        nloc = np.empty(n_sub, dtype=np.int64)
        check(mwi_decomposition(self.h, _ptr(part, C.c_int32), _ptr(nloc, C.c_int64)))
        return part, nloc

    def factor_stats(self):
        a, b, c = C.c_int64(), C.c_int64(), C.c_int64()
        d = C.c_double()
        check(mwi_factor_stats(self.h, C.byref(a), C.byref(b), C.byref(c), C.byref(d)))
        return dict(factor_entries=a.value, n_fronts=b.value, max_front=c.value, factor_flops=d.value)

    def device_bytes(self):
        """Device bytes held by this problem (the mesh's shared structures excluded)."""
        b = C.c_int64()
        check(mwi_problem_device_bytes(self.h, C.byref(b)))
        return b.value

    def oras_traffic(self, m):
        """Algorithmic bytes of one ORAS application to m columns."""
        b = C.c_double()
        check(mwi_oras_traffic(self.h, m, C.byref(b)))
        return b.value

    def kernel_times(self, reset=True):
        ms = np.zeros(4)
        cnt = np.zeros(4, dtype=np.int64)
        check(mwi_kernel_times(self.h, _ptr(ms, C.c_double), _ptr(cnt, C.c_int64), 1 if reset else 0))
        return ms, cnt

    def misfit(self, S_meas, w=None):
        Sm = np.ascontiguousarray(np.asarray(S_meas, dtype=np.complex128).T)
        wp = None
        if w is not None:
            wc = np.ascontiguousarray(np.asarray(w, dtype=np.float64).T)
            wp = _ptr(wc, C.c_double)
        J = C.c_double()
        check(mwi_misfit(self.h, _ptr(Sm.view(np.float64), C.c_double), wp, C.byref(J)))
        return J.value

    def close(self):
        if self.h:
            check(mwi_problem_destroy(self.h))
            self.h = None

    def __del__(self):
        try:
            if self.h:
                mwi_problem_destroy(self.h)
        except Exception:
            pass
