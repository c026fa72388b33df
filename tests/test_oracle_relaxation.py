"""Pins of transverse relaxation and per-compartment initial conditions
(Section 2, the T2 term of the Bloch-Torrey equation and the initial
condition; Section 3, "Initial conditions").  At g = 0 and kappa = 0 each
compartment keeps a spatially constant field, so the theta-scheme reduces to
the scalar recursion u^n = u^{n-1} (1 - (1-th) dt/T2) / (1 + th dt/T2):
S = sum_c rho_c |Omega_c| r_c^N exactly, with |Omega_c| summed from the
tetrahedron volumes (not from the oracle's assembly), tending to
exp(-TE/T2) at second order in dt."""

import numpy as np

import geom
import oracle


def _volumes(p):
    X = p.xyz[p.tets]
    v = np.abs(np.einsum("ij,ij->i", X[:, 1] - X[:, 0], np.cross(X[:, 2] - X[:, 0], X[:, 3] - X[:, 0]))) / 6.0
    return np.bincount(p.tet_cmpt, weights=v, minlength=p.n_cmpt)


def _case(dt, kappa=0.0):
    p = geom.cfg2(n=5, kappa=kappa, bvals=(0.0,), dt=dt)
    p.delta, p.Delta, p.TE = 1000.0, 1000.0, 2000.0
    p.inv_T2 = np.array([1.0 / 20000.0, 1.0 / 50000.0])[: p.n_cmpt]
    p.rho = np.array([1.0, 0.6])[: p.n_cmpt]
    return p


def test_relaxation_exact_discrete_product():
    p = _case(50.0)
    vol = _volumes(p)
    th, dt, N = p.theta, p.dt, p.n_steps
    r = (1 - (1 - th) * dt * p.inv_T2) / (1 + th * dt * p.inv_T2)
    want = float(np.sum(p.rho * vol * r ** N))
    S = oracle.run(p)[0]
    assert abs(S - want) < 1e-11 * want


def test_relaxation_tends_to_exponential():
    errs = []
    for dt in (100.0, 50.0):
        p = _case(dt)
        vol = _volumes(p)
        want = float(np.sum(p.rho * vol * np.exp(-p.TE * p.inv_T2)))
        errs.append(abs(oracle.run(p)[0].real - want) / want)
    assert 3.5 < errs[0] / errs[1] < 4.5


def test_exchange_conserves_total_initial_magnetization():
    """kappa > 0, g = 0, no relaxation: the permeable membranes move
    magnetization between compartments, but sum_c rho_c |Omega_c| is kept at
    every step (1^T (K + J) = 0)."""
    p = _case(50.0, kappa=1e-3)
    p.inv_T2 = None
    vol = _volumes(p)
    S, hist = oracle.run(p, return_history=True)
    total = float(np.sum(p.rho * vol))
    assert np.max(np.abs(hist[0] - total)) < 1e-10 * total


def test_three_layer_t2_orders_the_signals():
    """Section 4's T2 study on the three-layer cross-section: relaxation in any
    layer lowers every signal, more so where more magnetization sits (the two
    outer layers hold more area than the inner disk)."""
    S = {}
    for name, inv in (("none", (0.0, 0.0, 0.0)), ("inner", (1 / 40000.0, 0.0, 0.0)),
                      ("outer", (0.0, 1 / 40000.0, 1 / 40000.0))):
        p = geom.layered_disk(n=16, rho=(1.0, 1.0, 1.0), bvals=(0.0, 2000.0, 4000.0), dirs=((0.0, 1.0, 0.0),))
        p.delta, p.Delta, p.TE = 10000.0, 10000.0, 20000.0
        p.inv_T2 = np.array(inv)
        S[name] = oracle.run(p).real
    assert np.all(S["inner"] < S["none"]) and np.all(S["outer"] < S["none"])
    assert S["outer"][0] < S["inner"][0]
