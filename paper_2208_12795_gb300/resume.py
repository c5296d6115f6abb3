"""Checkpoint and resume of a particle run: the particle SoA, the accumulated
edge deposit G_cum and the step index in one file.

The paper keeps no such state on disk; this is the run-level counterpart of
the gradient window's in-memory checkpoints.  A resumed run continues
bit for bit in its particle state (every particle's step depends only on its
own state, the mesh and the envelope), and its G_cum continues from the saved
value; later sums may differ in the last bits from an uninterrupted run
because the device accumulates them with atomics.
"""
from __future__ import annotations

import numpy as np
import torch

from .env import FempicEnv, ParticleState

FORMAT = 1
_COLS = ("x", "y", "z", "vx", "vy", "vz", "tet", "status", "n_cross")


def save_run(path, env: FempicEnv, st: ParticleState, step: int, t: float, extra: dict | None = None):
    """Write the state after `step` steps (time t) to `path`.  A step deposit
    still pending in the env is first finalized into G_cum, as
    fempic_deposit would do; G_cum is read through fempic_accumulate."""
    dev = st.x.device
    dG = torch.empty(env.n_edges, dtype=torch.float64, device=dev)
    G = torch.empty(env.n_edges, dtype=torch.float64, device=dev)
    env.deposit_local(dG)
    env.accumulate(0.0, 0.0, dG, G_cum_out=G)
    rec = {
        "format": FORMAT,
        "precision": int(env.precision),
        "counts": [int(env.n_nodes), int(env.n_edges), int(env.n_faces), int(env.n_tets)],
        "step": int(step),
        "t": float(t),
        "species_begin": st.species_begin.copy(),
        "q": st.q.copy(), "m": st.m.copy(), "w": st.w.copy(),
        "G_cum": G.cpu(),
        "extra": dict(extra or {}),
    }
    for k in _COLS:
        v = getattr(st, k)
        rec[k] = None if v is None else v.cpu()
    torch.save(rec, path)


def load_run(path, env: FempicEnv, device="cuda"):
    """Read a file written by save_run into `env` (same mesh and precision):
    G_cum is set to the saved value (the env's deposit accumulators are
    reset first).  Returns (ParticleState on `device`, step, t, extra)."""
    rec = torch.load(path, map_location="cpu", weights_only=False)
    if rec.get("format") != FORMAT:
        raise ValueError(f"{path}: unknown checkpoint format {rec.get('format')!r}")
    counts = [int(env.n_nodes), int(env.n_edges), int(env.n_faces), int(env.n_tets)]
    if rec["counts"] != counts:
        raise ValueError(f"{path}: saved on a mesh with counts {rec['counts']}, env has {counts}")
    if rec["precision"] != int(env.precision):
        raise ValueError(f"{path}: saved in precision form {rec['precision']}, env uses {env.precision}")
    d = lambda k: None if rec[k] is None else rec[k].to(device)
    st = ParticleState(d("x"), d("y"), d("z"), d("vx"), d("vy"), d("vz"),
                       np.asarray(rec["species_begin"]), np.asarray(rec["q"]), np.asarray(rec["m"]),
                       np.asarray(rec["w"]), tet=d("tet"), track_crossings=rec["n_cross"] is not None)
    st.status = d("status")
    if rec["n_cross"] is not None:
        st.n_cross = d("n_cross")
    env.reset_deposit()
    env.accumulate(0.0, 0.0, rec["G_cum"].to(device))
    return st, rec["step"], rec["t"], rec["extra"]
