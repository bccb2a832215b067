"""Checkpoint files of the chunked MD driver round-trip on the host (no GPU)."""
import numpy as np

from paper_1708_01135_gb300 import mdrun
from paper_1708_01135_gb300 import workloads as W


def test_checkpoint_round_trip(tmp_path):
    pos, q, L = W.rocksalt(4, 1.0, 0.05, seed=1)
    st = mdrun.start(L, 1.1, 2.0, 6, "fp64", pos, q, dt=1e-3, vel=np.full((64, 3), 0.25))
    st["step"] = 17
    st["log"] = np.arange(18 * 6, dtype=np.float64).reshape(18, 6)
    path = str(tmp_path / "ck.npz")
    mdrun.save(st, path)
    back = mdrun.resume(path)
    for k, v in st.items():
        if isinstance(v, np.ndarray):
            assert np.array_equal(back[k], v), k
        else:
            assert back[k] == v and type(back[k]) is type(v), k
