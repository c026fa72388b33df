"""Failure handling on the GPU, with every fault made on the host side:
iteration caps, an RHS whose arithmetic overflows, and invalid calls.  No
test traps, faults or hangs the GPU: every device loop is bounded and a
frozen system simply stops."""
import numpy as np
import pytest

import geom

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bt():
    from paper_1908_01719_gb300 import build, bt as btmod
    build.build()
    return btmod


@pytest.fixture(scope="module")
def sim_cls(bt):
    from paper_1908_01719_gb300.simulate import Simulation
    return Simulation


@pytest.mark.parametrize("mode", ["plain", "mixed"])
def test_iteration_cap_reports_enoconv(sim_cls, bt, mode):
    p = geom.cfg2(n=6, kappa=1e-4, bvals=(1000.0, 3000.0))
    sim = sim_cls(p)
    try:
        m = bt.BT_MODE_PLAIN_FP64 if mode == "plain" else bt.BT_MODE_MIXED
        S, err, stat, st = sim.run(m, raise_on_status=False, max_iter=1, max_refine=1, tol_fp64=1e-14,
                                   tol_inner=1e-12, tol_ref=1e-14)
        assert st == bt.BT_ENOCONV
        assert np.all(stat == bt.BT_ENOCONV)
    finally:
        sim.close()


@pytest.mark.parametrize("mode", ["plain", "mixed"])
def test_overflowing_rhs_is_isolated(sim_cls, bt, mode):
    """One b-value so large that its arithmetic overflows: that RHS ends with
    BT_ENAN, the others finish with their normal signals."""
    p = geom.cfg2(n=6, kappa=1e-4, bvals=(1000.0, 1e308, 3000.0))
    good = geom.cfg2(n=6, kappa=1e-4, bvals=(1000.0, 3000.0))
    m = bt.BT_MODE_PLAIN_FP64 if mode == "plain" else bt.BT_MODE_MIXED
    sim = sim_cls(p)
    try:
        S, err, stat, st = sim.run(m, raise_on_status=False)
    finally:
        sim.close()
    sim = sim_cls(good)
    try:
        Sg, _, statg, _ = sim.run(m)
    finally:
        sim.close()
    assert st == bt.BT_ENAN and stat[1] == bt.BT_ENAN
    assert stat[0] == 0 and stat[2] == 0
    assert np.max(np.abs(S[[0, 2]] - Sg) / np.abs(Sg)) < 1e-9


def test_invalid_calls(sim_cls, bt):
    p = geom.cfg1(n=3)
    ctx = bt.bt_create(0)
    try:
        bt.bt_upload_mesh(ctx, p.xyz, p.tets, p.tet_cmpt, p.D_cmpt, p.kappa_cmpt, 0, p.box_lo, p.box_hi)
        with pytest.raises(bt.BtError) as e:
            bt.bt_run(ctx, bt.BT_MODE_MIXED)
        assert e.value.code == bt.BT_ESTATE
        for dt, th in [(0.0, 0.5), (-5.0, 0.5), (50.0, 0.0), (50.0, 1.5), (float("nan"), 0.5)]:
            with pytest.raises(bt.BtError) as e:
                bt.bt_assemble(ctx, dt, th, bt.BT_FRAME_LAB)
            assert e.value.code == bt.BT_EINVAL
        bt.bt_assemble(ctx, 50.0, 0.5, bt.BT_FRAME_LAB)
        with pytest.raises(bt.BtError) as e:
            bt.bt_set_sequence(ctx, bt.BT_PGSE, 2500.0, 5000.0, 7525.0)   # TE not a multiple of dt
        assert e.value.code == bt.BT_EINVAL
        with pytest.raises(bt.BtError) as e:
            bt.bt_set_sequence(ctx, bt.BT_PGSE, 2500.0, 2000.0, 7500.0)   # Delta < delta
        assert e.value.code == bt.BT_EINVAL
        bt.bt_set_sequence(ctx, bt.BT_PGSE, 2500.0, 5000.0, 7500.0)
        with pytest.raises(bt.BtError) as e:
            bt.bt_set_gradients(ctx, np.zeros((1, 3)), [1000.0])          # zero direction
        assert e.value.code == bt.BT_EINVAL
        with pytest.raises(bt.BtError) as e:
            bt.bt_set_gradients(ctx, np.eye(3)[:1], [-1.0])               # negative b
        assert e.value.code == bt.BT_EINVAL
    finally:
        bt.bt_destroy(ctx)
    q = geom.free_periodic_box(n=3, L=5.0)
    ctx = bt.bt_create(0)
    try:
        bt.bt_upload_mesh(ctx, q.xyz, q.tets, q.tet_cmpt, q.D_cmpt, q.kappa_cmpt, 7, q.box_lo, q.box_hi)
        with pytest.raises(bt.BtError) as e:
            bt.bt_assemble(ctx, 50.0, 0.5, bt.BT_FRAME_LAB)                # periodic needs the transformed frame
        assert e.value.code == bt.BT_EINVAL
    finally:
        bt.bt_destroy(ctx)
