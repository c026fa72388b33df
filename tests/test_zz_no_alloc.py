"""The allocation-free gradient entry point (for callers that cannot allocate
device memory: stream capture, framework-owned allocators, no-allocation
services) against the existing bt_precond_eval on the same samples, on two
calls in a row.  Collected last so a failure here leaves every other result
intact."""
import numpy as np
import pytest
import scipy.sparse as sp

import geom
from oracle import precond as pc

pytestmark = pytest.mark.gpu


def _samples(n, seed):
    rng = np.random.default_rng(seed)
    feat = np.stack([rng.uniform(20, 100, n), rng.uniform(0, 3e-4, n), rng.uniform(1e-3, 3e-3, n),
                     rng.uniform(1e-5, 1e-4, n), rng.uniform(0.3, 2.0, n)], axis=1).astype(np.float32)
    G, h = [], []
    for s in range(n):
        m = 10
        B = rng.normal(size=(m, m)) * 0.1
        A = np.eye(m) * 3 + B + B.T + 1j * 0.2 * np.diag(rng.normal(size=m))
        r = rng.normal(size=m) + 1j * rng.normal(size=m)
        g_, h_ = pc.gram_data(sp.csr_matrix(A), r)
        G.append(g_)
        h.append(h_)
    return feat, np.array(G), np.array(h)


def test_noalloc_gradient_matches_existing_entry_point():
    torch = pytest.importorskip("torch")
    from paper_1908_01719_gb300 import build, bt
    from paper_1908_01719_gb300.simulate import Simulation
    build.build()
    n = 96
    feat, G, h = _samples(n, 11)
    rng = np.random.default_rng(12)
    w = (rng.normal(size=bt.BT_PRECOND_NPARAM) * 0.2).astype(np.float32)
    sim = Simulation(geom.cfg1(n=2))
    try:
        bt.bt_load_precond(sim.ctx, w)
        _, loss_ref, grad_ref = bt.bt_precond_eval(sim.ctx, feat, G, h)
    finally:
        sim.close()
    dev = torch.device("cuda", 0)
    w_t = torch.tensor(w, device=dev)
    f_t = torch.tensor(feat, device=dev)
    G_t = torch.tensor(G.reshape(n, 81), dtype=torch.float32, device=dev)
    h_t = torch.tensor(h, dtype=torch.float32, device=dev)
    grad_t = torch.zeros(bt.BT_PRECOND_NPARAM, dtype=torch.float64, device=dev)
    loss_t = torch.zeros(n, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev).cuda_stream
    for call in range(2):
        grad_t.zero_()
        loss_t.zero_()
        st = bt.bt_precond_grad_noalloc(w_t.data_ptr(), n, f_t.data_ptr(), G_t.data_ptr(), h_t.data_ptr(),
                                        grad_t.data_ptr(), loss_t.data_ptr(), stream)
        assert st == bt.BT_OK
        torch.cuda.synchronize(dev)
        g = grad_t.cpu().numpy()
        assert np.linalg.norm(g - grad_ref) <= 1e-6 * np.linalg.norm(grad_ref), call
        assert abs(float(loss_t.double().mean()) - loss_ref) <= 1e-6 * abs(loss_ref), call
    # sizes beyond the fixed scratch are refused before any launch
    too_many = bt.BT_NOALLOC_MAX_SAMPLES + 1
    assert bt.bt_precond_grad_noalloc(w_t.data_ptr(), too_many, f_t.data_ptr(), G_t.data_ptr(), h_t.data_ptr(),
                                      grad_t.data_ptr(), loss_t.data_ptr(), stream) == bt.BT_EINVAL
