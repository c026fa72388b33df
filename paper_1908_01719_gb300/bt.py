"""Thin Python binding of libbtgpu (include/bt.h), argument marshalling only.

Every function has the name of the C entry point it calls.  Arrays are NumPy
arrays on the host; the library copies what it needs.  A non-zero status
raises BtError with the library's message.  The library must have been built
(``paper_1908_01719_gb300.build.build()``); there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbtgpu.so")

BT_OK, BT_EINVAL, BT_ENOMEM, BT_ECUDA, BT_ENOCONV, BT_ENAN, BT_ETIMEOUT, BT_ESTATE, BT_ENODEV = range(9)
BT_FRAME_LAB, BT_FRAME_TRANSFORMED = 0, 1
BT_PGSE = 0
# temporal profiles of bt_set_waveform / bt_waveform_tables
WAVEFORMS = {"pgse": 0, "double_pgse": 1, "cos_ogse": 2, "sin_ogse": 3, "trapezoid": 4, "double_trapezoid": 5}
BT_MODE_PLAIN_FP64, BT_MODE_MIXED, BT_MODE_LEARNED = 0, 1, 2
BT_OPT_RESID_FP64, BT_OPT_PROFILE, BT_OPT_NO_GRAPH = 1, 2, 4
BT_OPT_VARIANT_ROW, BT_OPT_VARIANT_HALO, BT_OPT_VARIANT_SLICE, BT_OPT_SLICE_ONE_STAGE = 8, 16, 32, 64
BT_OPT_SLICE_CONFIG_SHIFT = 8
# Krylov variants of bt_get_tuning: row, halo, then the four slice configurations
VARIANTS = ["row", "halo", "slice", "slice1", "slice_small", "slice_small1", "slice_ws"]


def slice_config_flag(c):
    """Option flags forcing slice configuration c (0..4)."""
    return (c + 1) << BT_OPT_SLICE_CONFIG_SHIFT
PLANES = {"M": 0, "K": 1, "J": 2, "MD": 3, "Mx": 4, "My": 5, "Mz": 6, "Ex": 7, "Ey": 8, "Ez": 9, "A0": 10,
          "MR": 11}

# every symbol include/bt.h declares
EXPORTS = ["bt_create", "bt_destroy", "bt_set_stream", "bt_last_error", "bt_upload_mesh", "bt_get_sizes",
           "bt_get_dofmap", "bt_get_pattern", "bt_assemble", "bt_get_plane", "bt_set_sequence",
           "bt_set_gradients", "bt_default_opts", "bt_run", "bt_get_signals", "bt_get_stats",
           "bt_train_default_opts", "bt_precond_features", "bt_collect_precond_data", "bt_train_precond",
           "bt_precond_eval", "bt_save_precond", "bt_load_precond", "bt_precond_grad_noalloc",
           "bt_set_segments", "bt_get_tuning", "bt_get_state", "bt_get_halo_tiles", "bt_set_profile", "bt_set_relaxation", "bt_set_diffusion_tensor", "bt_set_weak_periodic", "bt_upload_mesh_2d",
           "bt_upload_mesh_1d", "bt_upload_mesh_surface", "bt_set_element_tensors", "bt_waveform_tables",
           "bt_set_waveform", "bt_get_segment_stats", "bt_set_precond_poly", "bt_chebyshev_poly",
           "bt_fit_chebyshev", "bt_get_precond_stats"]
BT_NOALLOC_MAX_SAMPLES = 2048
BT_PRECOND_NPARAM = 5 * 64 + 64 + 64 * 64 + 64 + 9 * 64 + 9
BT_TRAIN_CONTINUE = 1


class BtError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"[bt status {code}] {msg}")
        self.code = code


class bt_solver_opts(C.Structure):
    _fields_ = [("tol_fp64", C.c_double), ("tol_inner", C.c_double), ("tol_ref", C.c_double),
                ("max_iter", C.c_int32), ("max_refine", C.c_int32), ("check_every", C.c_int32),
                ("flags", C.c_uint32), ("rhs_begin", C.c_int32), ("rhs_end", C.c_int32)]


class bt_train_opts(C.Structure):
    _fields_ = [("epochs", C.c_int32), ("batch", C.c_int32), ("lr", C.c_double), ("seed", C.c_uint64),
                ("flags", C.c_uint32), ("rel_err", C.c_double)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_1908_01719_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        P, I32, I64, U32, D = C.c_void_p, C.c_int32, C.c_int64, C.c_uint32, C.c_double
        sig = {
            "bt_create": [C.POINTER(P), C.c_int],
            "bt_destroy": [P],
            "bt_set_stream": [P, P],
            "bt_upload_mesh": [P, I64, P, I64, P, P, I32, P, P, U32, P, P],
            "bt_upload_mesh_2d": [P, I64, P, I64, P, P, I32, P, P, U32, P, P],
            "bt_upload_mesh_1d": [P, I64, P, I64, P, P, I32, P, P, P],
            "bt_upload_mesh_surface": [P, I64, P, I64, P, P, I32, P, P, P, P],
            "bt_set_element_tensors": [P, P],
            "bt_get_sizes": [P, P, P, P],
            "bt_get_dofmap": [P, P, P],
            "bt_get_pattern": [P, P, P],
            "bt_assemble": [P, D, D, U32],
            "bt_get_plane": [P, C.c_int, P],
            "bt_set_sequence": [P, C.c_int, D, D, D],
            "bt_set_gradients": [P, I32, P, I32, P],
            "bt_set_profile": [P, I32, P, D],
            "bt_waveform_tables": [C.c_int, D, D, D, D, I32, D, P, P, P],
            "bt_get_segment_stats": [P, I32, P],
            "bt_set_waveform": [P, C.c_int, D, D, D, I32, D],
            "bt_set_relaxation": [P, P, P],
            "bt_set_diffusion_tensor": [P, P],
            "bt_set_weak_periodic": [P, U32, D],
            "bt_set_segments": [P, I32, P, P, P, P],
            "bt_get_tuning": [P, P, P, P, P],
            "bt_default_opts": [C.POINTER(bt_solver_opts)],
            "bt_run": [P, C.c_int, C.POINTER(bt_solver_opts)],
            "bt_get_signals": [P, P, P, P],
            "bt_get_state": [P, I32, P, P],
            "bt_get_halo_tiles": [P, I32, P, P, P, P, P, P, P, P, P],
            "bt_get_stats": [P, P, P, P, P, P, P, P, P, P, P],
            "bt_train_default_opts": [C.POINTER(bt_train_opts)],
            "bt_precond_features": [P, P, P, P],
            "bt_collect_precond_data": [P, C.POINTER(bt_solver_opts), I32, P, P, P, P],
            "bt_train_precond": [P, I64, P, P, P, C.POINTER(bt_train_opts), P],
            "bt_precond_eval": [P, I64, P, P, P, D, P, P, P],
            "bt_save_precond": [P, P],
            "bt_load_precond": [P, P],
            "bt_precond_grad_noalloc": [P, I32, P, P, P, P, P, P],
            "bt_set_precond_poly": [P, P],
            "bt_chebyshev_poly": [D, D, P],
            "bt_fit_chebyshev": [I64, P, P, D, P, P, P, P],
            "bt_get_precond_stats": [P, P],
        }
        for name, args in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = C.c_int
        L.bt_last_error.argtypes = [P]
        L.bt_last_error.restype = C.c_char_p
        _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p)


def _check(ctx, st):
    if st != BT_OK:
        msg = lib().bt_last_error(ctx).decode() if ctx else ""
        raise BtError(st, msg)


def bt_create(device: int):
    h = C.c_void_p()
    st = lib().bt_create(C.byref(h), device)
    if st != BT_OK:
        raise BtError(st, f"bt_create(device={device}) failed")
    return h


def bt_destroy(ctx):
    lib().bt_destroy(ctx)


def bt_set_stream(ctx, stream_handle: int):
    _check(ctx, lib().bt_set_stream(ctx, C.c_void_p(stream_handle)))


def bt_last_error(ctx) -> str:
    return lib().bt_last_error(ctx).decode()


def bt_upload_mesh(ctx, xyz, tets, tet_cmpt, D_cmpt, kappa_cmpt, periodic_mask, box_lo, box_hi):
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    tets = np.ascontiguousarray(tets, dtype=np.int32)
    tc = np.ascontiguousarray(tet_cmpt, dtype=np.int32)
    D = np.ascontiguousarray(D_cmpt, dtype=np.float64)
    K = np.ascontiguousarray(kappa_cmpt, dtype=np.float64)
    lo = np.ascontiguousarray(box_lo, dtype=np.float64)
    hi = np.ascontiguousarray(box_hi, dtype=np.float64)
    _check(ctx, lib().bt_upload_mesh(ctx, len(xyz), _ptr(xyz), len(tets), _ptr(tets), _ptr(tc), len(D), _ptr(D),
                                     _ptr(K), int(periodic_mask), _ptr(lo), _ptr(hi)))


def bt_upload_mesh_2d(ctx, xy, tris, tri_cmpt, D_cmpt, kappa_cmpt, periodic_mask, box_lo, box_hi):
    """2-D mesh of counter-clockwise triangles in the xy plane."""
    xy = np.ascontiguousarray(np.asarray(xy, dtype=np.float64)[:, :2])
    tris = np.ascontiguousarray(tris, dtype=np.int32)
    tc = np.ascontiguousarray(tri_cmpt, dtype=np.int32)
    D = np.ascontiguousarray(D_cmpt, dtype=np.float64)
    K = np.ascontiguousarray(kappa_cmpt, dtype=np.float64)
    lo = np.ascontiguousarray(np.asarray(box_lo, dtype=np.float64)[:2])
    hi = np.ascontiguousarray(np.asarray(box_hi, dtype=np.float64)[:2])
    _check(ctx, lib().bt_upload_mesh_2d(ctx, len(xy), _ptr(xy), len(tris), _ptr(tris), _ptr(tc), len(D), _ptr(D),
                                        _ptr(K), int(periodic_mask), _ptr(lo), _ptr(hi)))


def bt_upload_mesh_1d(ctx, xyz, segs, seg_cmpt, D_cmpt, box_lo, box_hi):
    """1-D manifold: P1 segments (centre lines of thin tubes) embedded in 3-D."""
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    segs = np.ascontiguousarray(segs, dtype=np.int32)
    sc = np.ascontiguousarray(seg_cmpt, dtype=np.int32)
    D = np.ascontiguousarray(D_cmpt, dtype=np.float64)
    lo = np.ascontiguousarray(box_lo, dtype=np.float64)
    hi = np.ascontiguousarray(box_hi, dtype=np.float64)
    _check(ctx, lib().bt_upload_mesh_1d(ctx, len(xyz), _ptr(xyz), len(segs), _ptr(segs), _ptr(sc), len(D), _ptr(D),
                                        _ptr(lo), _ptr(hi)))


def bt_upload_mesh_surface(ctx, xyz, tris, tri_cmpt, D_cmpt, kappa_cmpt, box_lo, box_hi):
    """Thin layer: P1 triangles of a surface embedded in 3-D."""
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    tris = np.ascontiguousarray(tris, dtype=np.int32)
    tc = np.ascontiguousarray(tri_cmpt, dtype=np.int32)
    D = np.ascontiguousarray(D_cmpt, dtype=np.float64)
    K = np.ascontiguousarray(kappa_cmpt, dtype=np.float64)
    lo = np.ascontiguousarray(box_lo, dtype=np.float64)
    hi = np.ascontiguousarray(box_hi, dtype=np.float64)
    _check(ctx, lib().bt_upload_mesh_surface(ctx, len(xyz), _ptr(xyz), len(tris), _ptr(tris), _ptr(tc), len(D),
                                             _ptr(D), _ptr(K), _ptr(lo), _ptr(hi)))


def bt_get_sizes(ctx):
    a = (C.c_int64 * 3)()
    _check(ctx, lib().bt_get_sizes(ctx, C.byref(a, 0), C.byref(a, 8), C.byref(a, 16)))
    return int(a[0]), int(a[1]), int(a[2])


def bt_get_dofmap(ctx):
    n, _, _ = bt_get_sizes(ctx)
    dn = np.empty(n, np.int32)
    dc = np.empty(n, np.int32)
    _check(ctx, lib().bt_get_dofmap(ctx, _ptr(dn), _ptr(dc)))
    return dn, dc


def bt_get_pattern(ctx):
    n, nnz, _ = bt_get_sizes(ctx)
    rp = np.empty(n + 1, np.int64)
    col = np.empty(nnz, np.int32)
    _check(ctx, lib().bt_get_pattern(ctx, _ptr(rp), _ptr(col)))
    return rp, col


def bt_assemble(ctx, dt_us: float, theta: float, frame: int):
    _check(ctx, lib().bt_assemble(ctx, float(dt_us), float(theta), int(frame)))


def bt_get_plane(ctx, which):
    _, nnz, _ = bt_get_sizes(ctx)
    v = np.empty(nnz, np.float64)
    idx = PLANES[which] if isinstance(which, str) else int(which)
    _check(ctx, lib().bt_get_plane(ctx, idx, _ptr(v)))
    return v


def bt_set_sequence(ctx, kind, delta, Delta, TE):
    _check(ctx, lib().bt_set_sequence(ctx, int(kind), float(delta), float(Delta), float(TE)))


def bt_set_segments(ctx, node_off, delta, Delta, TE):
    no = np.ascontiguousarray(node_off, dtype=np.int64)
    d = np.ascontiguousarray(delta, dtype=np.float64)
    D = np.ascontiguousarray(Delta, dtype=np.float64)
    T = np.ascontiguousarray(TE, dtype=np.float64)
    _check(ctx, lib().bt_set_segments(ctx, len(no) - 1, _ptr(no), _ptr(d), _ptr(D), _ptr(T)))


def bt_set_relaxation(ctx, inv_T2=None, rho=None):
    """1/T2 (1/us) and initial magnetization per compartment; None keeps the default."""
    a = None if inv_T2 is None else np.ascontiguousarray(inv_T2, dtype=np.float64)
    b = None if rho is None else np.ascontiguousarray(rho, dtype=np.float64)
    _check(ctx, lib().bt_set_relaxation(ctx, None if a is None else _ptr(a), None if b is None else _ptr(b)))


def bt_set_weak_periodic(ctx, axes, kappa_e=0.0):
    """Artificial-permeability coupling of the box faces on the axes of the bit mask."""
    _check(ctx, lib().bt_set_weak_periodic(ctx, int(axes), float(kappa_e)))


def bt_set_diffusion_tensor(ctx, D6=None):
    """Per-compartment diffusion tensors [n_cmpt, 6] (xx, yy, zz, xy, yz, zx); None = isotropic."""
    if D6 is None:
        _check(ctx, lib().bt_set_diffusion_tensor(ctx, None))
        return
    a = np.ascontiguousarray(D6, dtype=np.float64).reshape(-1, 6)
    _check(ctx, lib().bt_set_diffusion_tensor(ctx, _ptr(a)))


def bt_set_element_tensors(ctx, D6=None):
    """Cell-based diffusion tensors [n_elem, 6] (xx, yy, zz, xy, yz, zx), one row
    per element in upload order; None removes them."""
    if D6 is None:
        _check(ctx, lib().bt_set_element_tensors(ctx, None))
        return
    a = np.ascontiguousarray(D6, dtype=np.float64).reshape(-1, 6)
    _check(ctx, lib().bt_set_element_tensors(ctx, _ptr(a)))


def bt_set_profile(ctx, F, int_F2):
    """Arbitrary temporal profile: F[n] = int_0^{n dt} f (us), int_F2 = int_0^TE F^2 (us^3)."""
    F = np.ascontiguousarray(F, dtype=np.float64).ravel()
    _check(ctx, lib().bt_set_profile(ctx, len(F) - 1, _ptr(F), float(int_F2)))


def bt_waveform_tables(kind, delta, Delta, TE, dt, n_periods=1, ramp=0.0):
    """(F[n_steps + 1], int_0^TE F^2) of a named profile (WAVEFORMS), from the
    library; no context or GPU needed."""
    k = WAVEFORMS[kind] if isinstance(kind, str) else int(kind)
    n = C.c_int32()
    st = lib().bt_waveform_tables(k, float(delta), float(Delta), float(TE), float(dt), int(n_periods),
                                  float(ramp or 0.0), C.byref(n), None, None)
    if st != BT_OK:
        raise BtError(st, "bt_waveform_tables: invalid profile parameters")
    F = np.zeros(n.value + 1)
    I = C.c_double()
    lib().bt_waveform_tables(k, float(delta), float(Delta), float(TE), float(dt), int(n_periods),
                             float(ramp or 0.0), C.byref(n), _ptr(F), C.byref(I))
    return F, I.value


def bt_set_waveform(ctx, kind, delta, Delta, TE, n_periods=1, ramp=0.0):
    k = WAVEFORMS[kind] if isinstance(kind, str) else int(kind)
    _check(ctx, lib().bt_set_waveform(ctx, k, float(delta), float(Delta), float(TE), int(n_periods),
                                      float(ramp or 0.0)))


def bt_set_gradients(ctx, dirs, bvals):
    d = np.ascontiguousarray(dirs, dtype=np.float64).reshape(-1, 3)
    b = np.ascontiguousarray(bvals, dtype=np.float64).ravel()
    _check(ctx, lib().bt_set_gradients(ctx, len(d), _ptr(d), len(b), _ptr(b)))


def bt_default_opts(**kw):
    o = bt_solver_opts()
    lib().bt_default_opts(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def bt_run(ctx, mode, opts=None, raise_on_status=True):
    o = opts if opts is not None else bt_default_opts()
    st = lib().bt_run(ctx, int(mode), C.byref(o))
    if st != BT_OK and (raise_on_status or st not in (BT_ENOCONV, BT_ENAN)):
        _check(ctx, st)
    return st


def bt_get_signals(ctx, R):
    S = np.empty(2 * R, np.float64)
    err = np.empty(R, np.float64)
    stat = np.empty(R, np.int32)
    _check(ctx, lib().bt_get_signals(ctx, _ptr(S), _ptr(err), _ptr(stat)))
    return S[0::2] + 1j * S[1::2], err, stat


def bt_get_state(ctx, system):
    """u^N of one system of the last run, complex FP64, in dof order."""
    n = C.c_int64(0)
    _check(ctx, lib().bt_get_state(ctx, int(system), None, C.byref(n)))
    u = np.empty(2 * n.value, np.float64)
    _check(ctx, lib().bt_get_state(ctx, int(system), _ptr(u), C.byref(n)))
    return u[0::2] + 1j * u[1::2]


def bt_get_halo_tiles(ctx, umax):
    """The halo tiles of the shared-memory Krylov apply, as numpy arrays."""
    nt, nh = C.c_int64(0), C.c_int64(0)
    _check(ctx, lib().bt_get_halo_tiles(ctx, int(umax), C.byref(nt), C.byref(nh), *([None] * 7)))
    n_dof, nnz, _ = bt_get_sizes(ctx)
    out = {"r0": np.empty(nt.value + 1, np.int32), "rows": np.empty(n_dof, np.int32),
           "rowe": np.empty(n_dof + 1, np.int32), "rowl": np.empty(n_dof, np.uint16),
           "u0": np.empty(nt.value + 1, np.int32), "ucol": np.empty(nh.value, np.uint32),
           "lidx": np.empty(nnz, np.uint16)}
    _check(ctx, lib().bt_get_halo_tiles(ctx, int(umax), C.byref(nt), C.byref(nh),
                                        *[_ptr(out[k]) for k in ("r0", "rows", "rowe", "rowl", "u0", "ucol",
                                                                 "lidx")]))
    return out


def bt_get_segment_stats(ctx, G):
    """Active systems summed over the last run's SpMM launches, per segment."""
    out = np.zeros(G, dtype=np.int64)
    _check(ctx, lib().bt_get_segment_stats(ctx, int(G), _ptr(out)))
    return out


def bt_get_stats(ctx):
    i = (C.c_int64 * 7)()
    d = (C.c_double * 3)()
    _check(ctx, lib().bt_get_stats(ctx, C.byref(i, 0), C.byref(i, 8), C.byref(i, 16), C.byref(i, 24),
                                   C.byref(d, 0), C.byref(d, 8), C.byref(i, 32), C.byref(i, 40), C.byref(i, 48),
                                   C.byref(d, 16)))
    return {"steps": i[0], "krylov_iters": i[1], "refine_passes": i[2], "spmm_launches": i[3],
            "spmm_ms": d[0], "resid_ms": d[1], "resid_launches": i[4], "kernel_launches": i[5],
            "sys_iters": i[6], "vec_ms": d[2]}


def bt_train_default_opts(**kw):
    o = bt_train_opts()
    lib().bt_train_default_opts(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def bt_precond_features(ctx):
    a = (C.c_double * 3)()
    _check(ctx, lib().bt_precond_features(ctx, C.byref(a, 0), C.byref(a, 8), C.byref(a, 16)))
    return float(a[0]), float(a[1]), float(a[2])


def bt_collect_precond_data(ctx, steps, R, opts=None):
    steps = np.ascontiguousarray(steps, dtype=np.int32)
    ns = len(steps) * R
    feat = np.zeros((ns, 5), np.float32)
    G = np.zeros((ns, 81), np.float64)
    h = np.zeros((ns, 9), np.float64)
    o = opts if opts is not None else bt_default_opts()
    _check(ctx, lib().bt_collect_precond_data(ctx, C.byref(o), len(steps), _ptr(steps), _ptr(feat), _ptr(G),
                                              _ptr(h)))
    return feat, G.reshape(ns, 9, 9), h


def bt_train_precond(ctx, feat, G, h, opts=None):
    feat = np.ascontiguousarray(feat, dtype=np.float32)
    G = np.ascontiguousarray(G, dtype=np.float64).reshape(len(feat), 81)
    h = np.ascontiguousarray(h, dtype=np.float64).reshape(len(feat), 9)
    o = opts if opts is not None else bt_train_default_opts()
    hist = np.zeros(o.epochs, np.float64)
    _check(ctx, lib().bt_train_precond(ctx, len(feat), _ptr(feat), _ptr(G), _ptr(h), C.byref(o), _ptr(hist)))
    return hist


def bt_precond_eval(ctx, feat, G=None, h=None, rel_err=0.0):
    feat = np.ascontiguousarray(feat, dtype=np.float32)
    n = len(feat)
    coef = np.zeros((n, 9), np.float64)
    loss = np.zeros(1, np.float64)
    grad = np.zeros(BT_PRECOND_NPARAM, np.float64)
    if G is None:
        _check(ctx, lib().bt_precond_eval(ctx, n, _ptr(feat), None, None, 0.0, _ptr(coef), None, None))
        return coef, None, None
    Gc = np.ascontiguousarray(G, dtype=np.float64).reshape(n, 81)
    hc = np.ascontiguousarray(h, dtype=np.float64).reshape(n, 9)
    _check(ctx, lib().bt_precond_eval(ctx, n, _ptr(feat), _ptr(Gc), _ptr(hc), float(rel_err), _ptr(coef),
                                      _ptr(loss), _ptr(grad)))
    return coef, float(loss[0]), grad


def bt_save_precond(ctx):
    w = np.zeros(BT_PRECOND_NPARAM, np.float32)
    _check(ctx, lib().bt_save_precond(ctx, _ptr(w)))
    return w


def bt_load_precond(ctx, w):
    w = np.ascontiguousarray(w, dtype=np.float32)
    assert len(w) == BT_PRECOND_NPARAM
    _check(ctx, lib().bt_load_precond(ctx, _ptr(w)))


def bt_set_precond_poly(ctx, c9):
    """Fixed polynomial coefficients for BT_MODE_LEARNED (None: back to the network)."""
    if c9 is None:
        _check(ctx, lib().bt_set_precond_poly(ctx, None))
        return
    c = np.ascontiguousarray(c9, dtype=np.float64)
    assert c.shape == (9,)
    _check(ctx, lib().bt_set_precond_poly(ctx, _ptr(c)))


def bt_chebyshev_poly(lo, hi):
    """Monomial coefficients c_0..c_8 of the degree-8 Chebyshev polynomial
    preconditioner on [lo, hi] (library host code, no context)."""
    c = np.zeros(9)
    st = lib().bt_chebyshev_poly(float(lo), float(hi), _ptr(c))
    if st != BT_OK:
        raise BtError(st, "bt_chebyshev_poly: need 0 < lo < hi")
    return c


def bt_fit_chebyshev(G, h, rel_err=1e-6):
    """(lo, hi, c9, mean loss) of the Chebyshev interval fitted to samples
    whose G and h are known to relative accuracy rel_err."""
    n = len(h)
    Gc = np.ascontiguousarray(G, dtype=np.float64).reshape(n, 81)
    hc = np.ascontiguousarray(h, dtype=np.float64).reshape(n, 9)
    lo, hi, loss = C.c_double(), C.c_double(), C.c_double()
    c = np.zeros(9)
    st = lib().bt_fit_chebyshev(n, _ptr(Gc), _ptr(hc), float(rel_err), C.byref(lo), C.byref(hi), _ptr(c),
                                C.byref(loss))
    if st != BT_OK:
        raise BtError(st, "bt_fit_chebyshev: bad samples")
    return lo.value, hi.value, c, loss.value


def bt_get_precond_stats(ctx):
    n = C.c_int64()
    _check(ctx, lib().bt_get_precond_stats(ctx, C.byref(n)))
    return {"horner_launches": n.value}


def bt_precond_grad_noalloc(w_ptr, n, feat_ptr, G_ptr, h_ptr, grad_ptr, loss_ptr, stream=0):
    """Device-pointer call of the allocation-free gradient (see include/bt.h);
    returns the status code."""
    V = C.c_void_p
    return lib().bt_precond_grad_noalloc(V(w_ptr), int(n), V(feat_ptr), V(G_ptr), V(h_ptr), V(grad_ptr),
                                         V(loss_ptr), V(stream))


def bt_get_tuning(ctx):
    v = C.c_int32()
    d = (C.c_double * len(VARIANTS))()
    rv = C.c_int32()
    dr = (C.c_double * 2)()
    _check(ctx, lib().bt_get_tuning(ctx, C.byref(v), d, C.byref(rv), dr))
    out = {"variant": VARIANTS[v.value]}
    out.update({f"ms_iter_{name}": d[k] for k, name in enumerate(VARIANTS)})
    out.update({"resid_variant": ["row", "halo"][rv.value], "ms_resid_row": dr[0], "ms_resid_halo": dr[1]})
    return out
