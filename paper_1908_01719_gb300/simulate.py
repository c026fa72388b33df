"""Convenience driver over the C ABI: upload a geometry, assemble, set the
sequence and gradients, run, read the signals.  Marshalling only; every step of
the method runs inside libbtgpu."""
from __future__ import annotations

from . import bt


class Simulation:
    """One context holding one geometry.  `geom` is any object with the fields
    xyz, tets, tet_cmpt, D_cmpt, kappa_cmpt, periodic_mask, box_lo, box_hi,
    dt, theta, delta, Delta, TE, dirs, bvals, transformed, and optionally a
    temporal `profile` ({"kind": one of bt.WAVEFORMS, "n_periods", "ramp"}; None =
    PGSE), per-compartment `inv_T2`
    (1/us) and initial magnetization `rho`, per-compartment `D_tensor` or
    per-element `D_tensor_elem` (lab frame) and
    `weak_periodic` (lab frame)."""

    def __init__(self, geom, device: int = 0, stream: int | None = None):
        self.g = geom
        self.ctx = bt.bt_create(device)
        if stream is not None:
            bt.bt_set_stream(self.ctx, stream)
        if geom.tets.shape[1] == 2:
            bt.bt_upload_mesh_1d(self.ctx, geom.xyz, geom.tets, geom.tet_cmpt, geom.D_cmpt, geom.box_lo, geom.box_hi)
        elif getattr(geom, "surface", False):
            bt.bt_upload_mesh_surface(self.ctx, geom.xyz, geom.tets, geom.tet_cmpt, geom.D_cmpt, geom.kappa_cmpt,
                                      geom.box_lo, geom.box_hi)
        else:
            upload = bt.bt_upload_mesh_2d if geom.tets.shape[1] == 3 else bt.bt_upload_mesh
            upload(self.ctx, geom.xyz, geom.tets, geom.tet_cmpt, geom.D_cmpt, geom.kappa_cmpt,
                   geom.periodic_mask, geom.box_lo, geom.box_hi)
        self.n_dof, self.nnz, self.n_iface = bt.bt_get_sizes(self.ctx)
        self.frame = bt.BT_FRAME_TRANSFORMED if (geom.transformed or geom.periodic_mask) else bt.BT_FRAME_LAB
        seg = getattr(geom, "segments", None)
        self.G = 1 if seg is None else len(seg["node_off"]) - 1
        inv_T2, rho = getattr(geom, "inv_T2", None), getattr(geom, "rho", None)
        if inv_T2 is not None or rho is not None:
            bt.bt_set_relaxation(self.ctx, inv_T2, rho)
        if getattr(geom, "D_tensor", None) is not None:
            bt.bt_set_diffusion_tensor(self.ctx, geom.D_tensor)
        De = getattr(geom, "D_tensor_elem", None)
        if De is not None:
            if len(De) != len(geom.tets):
                raise ValueError("D_tensor_elem needs one row per element")
            bt.bt_set_element_tensors(self.ctx, De)
        weak = getattr(geom, "weak_periodic", None)
        if weak:
            bt.bt_set_weak_periodic(self.ctx, weak["axes"], weak.get("kappa_e") or 0.0)
        if device >= 0:
            bt.bt_assemble(self.ctx, geom.dt, geom.theta, self.frame)
            prof = getattr(geom, "profile", None)
            if seg is None and prof:
                bt.bt_set_waveform(self.ctx, prof["kind"], geom.delta, geom.Delta, geom.TE,
                                   prof.get("n_periods", 1), prof.get("ramp") or 0.0)
            elif seg is None:
                bt.bt_set_sequence(self.ctx, bt.BT_PGSE, geom.delta, geom.Delta, geom.TE)
            else:
                bt.bt_set_segments(self.ctx, seg["node_off"], seg["delta"], seg["Delta"], seg["TE"])
            bt.bt_set_gradients(self.ctx, geom.dirs, geom.bvals)
        self.R = len(geom.dirs) * len(geom.bvals)

    def run(self, mode=bt.BT_MODE_MIXED, raise_on_status=True, **opts):
        o = bt.bt_default_opts(**opts)
        st = bt.bt_run(self.ctx, mode, o, raise_on_status=raise_on_status)
        S, err, stat = bt.bt_get_signals(self.ctx, self.G * self.R)
        return S, err, stat, st

    def stats(self):
        return bt.bt_get_stats(self.ctx)

    def close(self):
        if self.ctx:
            bt.bt_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def simulate(geom, mode=bt.BT_MODE_MIXED, device: int = 0, **opts):
    sim = Simulation(geom, device)
    try:
        S, err, stat, _ = sim.run(mode, **opts)
        return S, err, stat
    finally:
        sim.close()
