"""CPU tests of the C ABI: the library loads, exports every declared entry
point, and its host pipeline (validation, periodic identification, interface
doubling, interface faces, CSR pattern) agrees with the oracle's own
construction.  Host-only contexts (device = -1) make no GPU call."""
import math
import os
import re

import numpy as np
import pytest

import geom
from oracle import btoracle as bo

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bt():
    from paper_1908_01719_gb300 import build, bt as btmod
    build.build()
    return btmod


def header_symbols():
    txt = open(os.path.join(ROOT, "include", "bt.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(bt_[a-z_0-9]+)\s*\(", txt)))


def test_exports_every_declared_symbol(bt):
    L = bt.lib()
    syms = header_symbols()
    assert len(syms) >= 16
    for s in syms:
        assert hasattr(L, s), s
    assert sorted(bt.EXPORTS) == syms


def test_gpu_calls_refused_on_host_only_context(bt):
    p = geom.cfg1(n=2)
    ctx = bt.bt_create(-1)
    try:
        bt.bt_upload_mesh(ctx, p.xyz, p.tets, p.tet_cmpt, p.D_cmpt, p.kappa_cmpt, 0, p.box_lo, p.box_hi)
        with pytest.raises(bt.BtError) as e:
            bt.bt_assemble(ctx, 50.0, 0.5, bt.BT_FRAME_LAB)
        assert e.value.code == bt.BT_ENODEV
    finally:
        bt.bt_destroy(ctx)


def _host(bt, p):
    ctx = bt.bt_create(-1)
    if p.tets.shape[1] == 2:
        bt.bt_upload_mesh_1d(ctx, p.xyz, p.tets, p.tet_cmpt, p.D_cmpt, p.box_lo, p.box_hi)
    elif p.surface:
        bt.bt_upload_mesh_surface(ctx, p.xyz, p.tets, p.tet_cmpt, p.D_cmpt, p.kappa_cmpt, p.box_lo, p.box_hi)
    else:
        up = bt.bt_upload_mesh_2d if p.tets.shape[1] == 3 else bt.bt_upload_mesh
        up(ctx, p.xyz, p.tets, p.tet_cmpt, p.D_cmpt, p.kappa_cmpt, p.periodic_mask, p.box_lo, p.box_hi)
    return ctx


def _oracle_pattern(a):
    S = (abs(a["M"]) + abs(a["J"]) + abs(a["Mx"])).tocsr()
    S.sort_indices()
    # structural union of the tet pattern and the face pattern
    Mst = a["M"].copy(); Mst.data[:] = 1
    Jst = a["J"].copy(); Jst.data[:] = 1
    U = (Mst + Jst).tocsr()
    U.sort_indices()
    return U.indptr, U.indices


@pytest.mark.parametrize("maker", [lambda: geom.cfg2(n=6, kappa=1e-4),
                                   lambda: geom.cfg3(n=8, n_dir=2, n_b=1),
                                   lambda: geom.cfg4(n=8, n_dir=1, bvals=(1000.0,))])
def test_doubling_faces_and_pattern_match_oracle(bt, maker):
    p = maker()
    a = bo.assemble(p)
    ctx = _host(bt, p)
    try:
        n, nnz, nf = bt.bt_get_sizes(ctx)
        assert n == a["n"]
        assert nf == a["n_iface"]
        dn, dc = bt.bt_get_dofmap(ctx)
        assert np.array_equal(dn, a["dof_node"]) and np.array_equal(dc, a["dof_cmpt"])
        rp, col = bt.bt_get_pattern(ctx)
        orp, ocol = _oracle_pattern(a)
        assert np.array_equal(rp, orp) and np.array_equal(col, ocol)
    finally:
        bt.bt_destroy(ctx)


def test_periodic_identification_counts(bt):
    p = geom.free_periodic_box(n=5, L=7.0)
    ctx = _host(bt, p)
    try:
        n, nnz, nf = bt.bt_get_sizes(ctx)
        assert n == 125 and nf == 0
        rp, col = bt.bt_get_pattern(ctx)
        assert np.all(np.diff(rp) == 15)    # Kuhn stencil, every node interior when periodic
    finally:
        bt.bt_destroy(ctx)


@pytest.mark.parametrize("defect", ["inverted", "node_range", "cmpt_range", "nan_kappa", "bad_box",
                                    "touching_free_cmpts", "neg_D"])
def test_mesh_validation_errors(bt, defect):
    p = geom.cfg2(n=3, kappa=1e-4)
    xyz, tets, tc = p.xyz.copy(), p.tets.copy(), p.tet_cmpt.copy()
    D, K, lo, hi = p.D_cmpt.copy(), p.kappa_cmpt.copy(), p.box_lo.copy(), p.box_hi.copy()
    if defect == "inverted":
        tets[5, [2, 3]] = tets[5, [3, 2]]
    elif defect == "node_range":
        tets[3, 1] = len(xyz)
    elif defect == "cmpt_range":
        tc[7] = 2
    elif defect == "nan_kappa":
        K[1] = math.nan
    elif defect == "bad_box":
        hi[0] = lo[0]
    elif defect == "touching_free_cmpts":
        tc = geom.label_sphere(xyz, tets, np.zeros(3), 5.0)
        K = np.array([math.inf, math.inf])
    elif defect == "neg_D":
        D[0] = -1.0
    ctx = bt.bt_create(-1)
    try:
        with pytest.raises(bt.BtError) as e:
            bt.bt_upload_mesh(ctx, xyz, tets, tc, D, K, 0, lo, hi)
        assert e.value.code == bt.BT_EINVAL
        assert len(bt.bt_last_error(ctx)) > 0
    finally:
        bt.bt_destroy(ctx)


def test_state_errors(bt):
    ctx = bt.bt_create(-1)
    try:
        with pytest.raises(bt.BtError) as e:
            bt.bt_get_sizes(ctx)
        assert e.value.code == bt.BT_ESTATE
        with pytest.raises(bt.BtError) as e:
            bt.bt_run(ctx, bt.BT_MODE_MIXED)
        assert e.value.code == bt.BT_ENODEV
    finally:
        bt.bt_destroy(ctx)


@pytest.mark.parametrize("maker,umax", [(lambda: geom.cfg2(n=10, kappa=1e-4), 96),
                                        (lambda: geom.cfg3(n=10, n_dir=1, n_b=1), 192),
                                        (lambda: geom.cfg4(n=12, n_dir=1, bvals=(1000.0,)), 384),
                                        (lambda: geom.square_disk(n=24, L=10.0, R=3.0), 96),
                                        (lambda: geom.dendrite_tree(seed=3, n_stems=3, depth=3), 96),
                                        (lambda: geom.spherical_shell(level=3, R=5.0, kappa=1e-4), 96)])
def test_halo_tiles_cover_the_pattern(bt, maker, umax):
    """Every row is owned by exactly one tile (at most 128 rows and 448 entries
    per tile); each tile's halo is the sorted,
    duplicate-free union of its rows' columns, within umax; the local indices
    of every entry point back to the CSR column; the owned flags mark exactly
    the tile's rows; and the halo is smaller than one gather per nonzero."""
    p = maker()
    ctx = _host(bt, p)
    try:
        rp, col = bt.bt_get_pattern(ctx)
        n = len(rp) - 1
        t = bt.bt_get_halo_tiles(ctx, umax)
        assert np.array_equal(np.sort(t["rows"]), np.arange(n))
        nt = len(t["r0"]) - 1
        assert t["r0"][0] == 0 and t["r0"][-1] == n and t["u0"][-1] == len(t["ucol"])
        for k in range(nt):
            rows = t["rows"][t["r0"][k]:t["r0"][k + 1]]
            assert 0 < len(rows) <= 128
            assert t["rowe"][t["r0"][k + 1]] - t["rowe"][t["r0"][k]] <= 448
            uc = t["ucol"][t["u0"][k]:t["u0"][k + 1]]
            ids = (uc & 0x7FFFFFFF).astype(np.int64)
            own = (uc >> 31).astype(bool)
            assert len(uc) <= umax
            assert np.all(np.diff(ids) > 0)
            want = np.unique(np.concatenate([col[rp[r]:rp[r + 1]] for r in rows]))
            assert np.array_equal(ids, want)
            assert np.array_equal(np.sort(ids[own]), np.sort(rows))
            for j, r in enumerate(rows):
                kk = t["r0"][k] + j
                e0, e1 = t["rowe"][kk], t["rowe"][kk + 1]
                assert e1 - e0 == rp[r + 1] - rp[r]
                assert np.array_equal(ids[t["lidx"][e0:e1]], col[rp[r]:rp[r + 1]])
                assert ids[t["rowl"][kk]] == r and own[t["rowl"][kk]]
        assert t["rowe"][-1] == len(col)
        assert len(t["ucol"]) < 0.5 * len(col)
        with pytest.raises(bt.BtError):
            bt.bt_get_halo_tiles(ctx, 8)
    finally:
        bt.bt_destroy(ctx)


def _host2d(bt, p):
    ctx = bt.bt_create(-1)
    bt.bt_upload_mesh_2d(ctx, p.xyz, p.tets, p.tet_cmpt, p.D_cmpt, p.kappa_cmpt, p.periodic_mask, p.box_lo,
                         p.box_hi)
    return ctx


@pytest.mark.parametrize("maker", [lambda: geom.square_disk(n=10, L=10.0, R=3.0),
                                   lambda: geom.free_periodic_square(n=5, L=6.0)])
def test_triangle_doubling_and_pattern_match_oracle(bt, maker):
    """2-D: interface edges doubled, dof map and CSR pattern as the oracle's."""
    p = maker()
    a = bo.assemble(p)
    ctx = _host2d(bt, p)
    try:
        n, nnz, nf = bt.bt_get_sizes(ctx)
        assert n == a["n"] and nf == a["n_iface"]
        dn, dc = bt.bt_get_dofmap(ctx)
        assert np.array_equal(dn, a["dof_node"]) and np.array_equal(dc, a["dof_cmpt"])
        rp, col = bt.bt_get_pattern(ctx)
        orp, ocol = _oracle_pattern(a)
        assert np.array_equal(rp, orp) and np.array_equal(col, ocol)
    finally:
        bt.bt_destroy(ctx)


def test_triangle_validation_and_refusals(bt):
    p = geom.square_disk(n=4, L=10.0, R=3.0)
    ctx = bt.bt_create(-1)
    try:
        tris = p.tets.copy()
        tris[2, [1, 2]] = tris[2, [2, 1]]                      # clockwise
        with pytest.raises(bt.BtError) as e:
            bt.bt_upload_mesh_2d(ctx, p.xyz, tris, p.tet_cmpt, p.D_cmpt, p.kappa_cmpt, 0, p.box_lo, p.box_hi)
        assert e.value.code == bt.BT_EINVAL
        with pytest.raises(bt.BtError) as e:                    # no z axis to identify in 2-D
            bt.bt_upload_mesh_2d(ctx, p.xyz, p.tets, p.tet_cmpt, p.D_cmpt, p.kappa_cmpt, 4, p.box_lo, p.box_hi)
        assert e.value.code == bt.BT_EINVAL
        bt.bt_upload_mesh_2d(ctx, p.xyz, p.tets, p.tet_cmpt, p.D_cmpt, p.kappa_cmpt, 0, p.box_lo, p.box_hi)
        bt.bt_set_weak_periodic(ctx, 3, 0.0)                    # boundary edges on the x and y sides
        with pytest.raises(bt.BtError) as e:                    # no z sides in 2-D
            bt.bt_set_weak_periodic(ctx, 4, 0.0)
        assert e.value.code == bt.BT_EINVAL
        xyz = p.xyz.copy()
        on_hi = np.flatnonzero(np.abs(xyz[:, 0] - p.box_hi[0]) < 1e-9)
        xyz[on_hi[1], 1] += 0.3 * (xyz[on_hi[2], 1] - xyz[on_hi[1], 1])   # sides no longer match
        bt.bt_upload_mesh_2d(ctx, xyz, p.tets, p.tet_cmpt, p.D_cmpt, p.kappa_cmpt, 0, p.box_lo, p.box_hi)
        bt.bt_set_weak_periodic(ctx, 2, 0.0)                    # y sides still match
        bt.bt_set_weak_periodic(ctx, 1, 0.0)                    # x sides coupled by projection
    finally:
        bt.bt_destroy(ctx)


def test_manifold_dofmap_and_pattern_match_oracle(bt):
    """1-D: one dof per node, tridiagonal along branches, wider at branch points."""
    p = geom.dendrite_tree(seed=2, n_stems=3, depth=3, length=(6.0, 12.0))
    a = bo.assemble(p)
    ctx = bt.bt_create(-1)
    try:
        bt.bt_upload_mesh_1d(ctx, p.xyz, p.tets, p.tet_cmpt, p.D_cmpt, p.box_lo, p.box_hi)
        n, nnz, nf = bt.bt_get_sizes(ctx)
        assert n == a["n"] == len(p.xyz) and nf == 0
        dn, dc = bt.bt_get_dofmap(ctx)
        assert np.array_equal(dn, a["dof_node"]) and np.array_equal(dc, a["dof_cmpt"])
        rp, col = bt.bt_get_pattern(ctx)
        orp, ocol = _oracle_pattern(a)
        assert np.array_equal(rp, orp) and np.array_equal(col, ocol)
        deg = np.bincount(p.tets.ravel(), minlength=len(p.xyz))
        assert np.array_equal(np.diff(rp), deg + 1)
    finally:
        bt.bt_destroy(ctx)


@pytest.mark.parametrize("defect", ["zero_length", "touching_cmpts", "node_range"])
def test_manifold_validation_errors(bt, defect):
    p = geom.line_segments(8)
    xyz, segs, sc, D = p.xyz.copy(), p.tets.copy(), p.tet_cmpt.copy(), p.D_cmpt.copy()
    if defect == "zero_length":
        xyz[3] = xyz[2]
    elif defect == "touching_cmpts":
        sc[4:] = 1
        D = np.array([2e-3, 1e-3])
    elif defect == "node_range":
        segs[2, 1] = len(xyz)
    ctx = bt.bt_create(-1)
    try:
        with pytest.raises(bt.BtError) as e:
            bt.bt_upload_mesh_1d(ctx, xyz, segs, sc, D, p.box_lo, p.box_hi)
        assert e.value.code == bt.BT_EINVAL
        assert len(bt.bt_last_error(ctx)) > 0
        bt.bt_upload_mesh_1d(ctx, p.xyz, p.tets, p.tet_cmpt, p.D_cmpt, p.box_lo, p.box_hi)
        with pytest.raises(bt.BtError) as e:
            bt.bt_set_weak_periodic(ctx, 1, 0.0)
        assert e.value.code == bt.BT_EINVAL
    finally:
        bt.bt_destroy(ctx)


def test_surface_dofmap_and_pattern_match_oracle(bt):
    """Thin layer: a sphere with a permeable cap, membrane along a latitude."""
    p = geom.spherical_shell(level=3, R=5.0, kappa=1e-4, cap_z=0.3)
    a = bo.assemble(p)
    ctx = bt.bt_create(-1)
    try:
        bt.bt_upload_mesh_surface(ctx, p.xyz, p.tets, p.tet_cmpt, p.D_cmpt, p.kappa_cmpt, p.box_lo, p.box_hi)
        n, nnz, nf = bt.bt_get_sizes(ctx)
        assert n == a["n"] and nf == a["n_iface"] > 0
        dn, dc = bt.bt_get_dofmap(ctx)
        assert np.array_equal(dn, a["dof_node"]) and np.array_equal(dc, a["dof_cmpt"])
        rp, col = bt.bt_get_pattern(ctx)
        orp, ocol = _oracle_pattern(a)
        assert np.array_equal(rp, orp) and np.array_equal(col, ocol)
        with pytest.raises(bt.BtError) as e:
            bt.bt_set_weak_periodic(ctx, 1, 0.0)
        assert e.value.code == bt.BT_EINVAL
        # any orientation is accepted; a zero-area triangle is not
        tris = p.tets.copy()
        tris[::2] = tris[::2, ::-1]
        bt.bt_upload_mesh_surface(ctx, p.xyz, tris, p.tet_cmpt, p.D_cmpt, p.kappa_cmpt, p.box_lo, p.box_hi)
        tris[5, 2] = tris[5, 1]
        with pytest.raises(bt.BtError) as e:
            bt.bt_upload_mesh_surface(ctx, p.xyz, tris, p.tet_cmpt, p.D_cmpt, p.kappa_cmpt, p.box_lo, p.box_hi)
        assert e.value.code == bt.BT_EINVAL
    finally:
        bt.bt_destroy(ctx)


def test_oversize_counts_refused_before_reading(bt):
    """Element and node counts beyond the 32-bit index limits are refused
    before any caller array is read (the arrays here are tiny)."""
    import ctypes as C
    p = geom.cfg1(n=2)
    xyz = np.ascontiguousarray(p.xyz)
    tets = np.ascontiguousarray(p.tets, dtype=np.int32)
    tc = np.ascontiguousarray(p.tet_cmpt, dtype=np.int32)
    D, K = np.ascontiguousarray(p.D_cmpt), np.ascontiguousarray(p.kappa_cmpt)
    lo, hi = np.ascontiguousarray(p.box_lo), np.ascontiguousarray(p.box_hi)
    ptr = lambda a: a.ctypes.data_as(C.c_void_p)
    L = bt.lib()
    ctx = bt.bt_create(-1)
    try:
        for nn, nt in [(1 << 31, len(tets)), (len(xyz), 1 << 28), (1 << 40, 1 << 40), (len(xyz), 1 << 60)]:
            st = L.bt_upload_mesh(ctx, nn, ptr(xyz), nt, ptr(tets), ptr(tc), 1, ptr(D), ptr(K), 0, ptr(lo), ptr(hi))
            assert st == bt.BT_EINVAL
            st = L.bt_upload_mesh_2d(ctx, nn, ptr(xyz), nt, ptr(tets), ptr(tc), 1, ptr(D), ptr(K), 0, ptr(lo),
                                     ptr(hi))
            assert st == bt.BT_EINVAL
        assert "32-bit" in bt.bt_last_error(ctx) or "invalid" in bt.bt_last_error(ctx)
    finally:
        bt.bt_destroy(ctx)


def test_element_tensor_validation(bt):
    p = geom.cfg2(n=3, kappa=1e-4)
    ctx = _host(bt, p)
    try:
        D = np.tile([2e-3, 1e-3, 1.5e-3, 1e-4, 0.0, -2e-4], (len(p.tets), 1))
        bt.bt_set_element_tensors(ctx, D)
        bt.bt_set_element_tensors(ctx, None)
        D[17] = [1e-3, 1e-3, 1e-3, 2e-3, 0.0, 0.0]              # |xy| > sqrt(xx yy): indefinite
        with pytest.raises(bt.BtError) as e:
            bt.bt_set_element_tensors(ctx, D)
        assert e.value.code == bt.BT_EINVAL and "17" in bt.bt_last_error(ctx)
        D[17, 3] = np.nan
        with pytest.raises(bt.BtError):
            bt.bt_set_element_tensors(ctx, D)
    finally:
        bt.bt_destroy(ctx)
