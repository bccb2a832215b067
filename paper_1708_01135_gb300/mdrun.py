"""Velocity-Verlet MD in chunks with checkpoints between them (stop and resume a long run).

Each chunk is one ewald_md call on the device; between chunks the state (positions,
velocities, step count) and everything needed to rebuild the plan (box, splitting parameter,
cutoffs, precision, time step, charges, masses) are written to an .npz file on the host.
Every ewald_md call starts by evaluating the forces at its starting positions, which is
exactly what the step before the boundary of an uninterrupted run evaluated last, and the
evaluation is deterministic, so a resumed run continues the same trajectory bit for bit.

    from paper_1708_01135_gb300 import mdrun
    st = mdrun.start(L, beta, r_c, k_max, "mixed", pos, q, dt=1e-3)
    st = mdrun.advance(st, 1000, chunk=100, checkpoint="run.npz")
    st = mdrun.resume("run.npz")            # later, in another process
    st = mdrun.advance(st, 1000, chunk=100, checkpoint="run.npz")
"""
from __future__ import annotations

import os

import numpy as np

from .ewald import MD_RECORD, Ewald

_KEYS = ("L", "beta", "r_c", "k_max", "precision", "dt", "step", "pos", "vel", "q", "mass",
         "log")


def start(L, beta, r_c, k_max, precision, pos, q, dt, vel=None, mass=None) -> dict:
    """A run at step 0 (host arrays; velocities default to zero, masses to one)."""
    pos = np.array(pos, dtype=np.float64)
    n = len(pos)
    return {"L": float(L), "beta": float(beta), "r_c": float(r_c), "k_max": int(k_max),
            "precision": str(precision), "dt": float(dt), "step": 0, "pos": pos,
            "vel": np.zeros((n, 3)) if vel is None else np.array(vel, dtype=np.float64),
            "q": np.array(q, dtype=np.float64),
            "mass": np.ones(n) if mass is None else np.array(mass, dtype=np.float64),
            "log": np.zeros((0, MD_RECORD))}


def save(state: dict, path: str) -> None:
    """Write the state to `path` (.npz), atomically: a temporary file, flushed to disk, then a
    rename, then the directory entry flushed, so that after a crash `path` holds either the
    previous checkpoint or this one in full."""
    tmp = path + ".tmp.npz"
    with open(tmp, "wb") as f:
        np.savez(f, **{k: np.asarray(state[k]) for k in _KEYS})
        f.flush()
        os.fsync(f.fileno())
    os.replace(tmp, path)
    try:
        fd = os.open(os.path.dirname(os.path.abspath(path)), os.O_RDONLY)
    except OSError:
        return
    try:
        os.fsync(fd)
    except OSError:
        pass
    finally:
        os.close(fd)


def resume(path: str) -> dict:
    """The state saved at `path`."""
    with np.load(path) as z:
        st = {k: z[k] for k in _KEYS}
    for k in ("L", "beta", "r_c", "dt"):
        st[k] = float(st[k])
    st["k_max"] = int(st["k_max"])
    st["step"] = int(st["step"])
    st["precision"] = str(st["precision"])
    return st


def advance(state: dict, steps: int, chunk: int = 100, checkpoint: str | None = None,
            device: str = "cuda") -> dict:
    """Advance the run by `steps` steps, `chunk` steps per ewald_md call, saving the state to
    `checkpoint` after every chunk.  Returns the new state; its log gains one record per
    step (E_real, E_recip, E_self, E_pot, E_kin, E_total after that step; the first record
    of a run is its initial state)."""
    import torch
    if steps < 0 or chunk < 1:
        raise ValueError("steps must be >= 0 and chunk >= 1")
    st = dict(state)
    dev = torch.device(device)
    tp = torch.tensor(st["pos"], device=dev)
    tv = torch.tensor(st["vel"], device=dev)
    tq = torch.tensor(st["q"], device=dev)
    tm = torch.tensor(st["mass"], device=dev)
    F = torch.empty_like(tp)
    logs = [np.asarray(st["log"]).reshape(-1, MD_RECORD)]
    with Ewald(st["L"], st["beta"], st["r_c"], st["k_max"], st["precision"]) as ew:
        done = 0
        while done < steps:
            k = min(chunk, steps - done)
            lg = torch.empty((k + 1, MD_RECORD), dtype=torch.float64, device=dev)
            ew.md(tp, tv, tq, F, st["dt"], k, mass=tm, log=lg)
            status = ew.status()
            if status != 0:
                raise RuntimeError(f"ewald_md reported status {status}")
            lg = lg.cpu().numpy()
            logs.append(lg if st["step"] == 0 and done == 0 and len(logs[0]) == 0 else lg[1:])
            done += k
            st["step"] += k
            st["pos"] = tp.cpu().numpy()
            st["vel"] = tv.cpu().numpy()
            st["log"] = np.concatenate(logs)
            if checkpoint:
                save(st, checkpoint)
    return st
