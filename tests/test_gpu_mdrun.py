"""MD in chunks with checkpoints (paper_1708_01135_gb300.mdrun): a run that stops at a
checkpoint and resumes from the file, with a fresh plan, continues the uninterrupted
trajectory bit for bit (positions, velocities and the energy log)."""
import numpy as np
import pytest

from gpu_common import need_gpu

from paper_1708_01135_gb300 import mdrun
from paper_1708_01135_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_resumed_run_continues_bit_for_bit(tmp_path, precision):
    need_gpu()
    pos, q, L = W.rocksalt(8, 1.0, 0.05, seed=3)
    st0 = mdrun.start(L, 1.0, 4.0, 10, precision, pos, q, dt=2e-3)
    whole = mdrun.advance(st0, 40, chunk=40)
    path = str(tmp_path / "run.npz")
    part = mdrun.advance(st0, 20, chunk=7, checkpoint=path)
    back = mdrun.resume(path)
    assert back["step"] == 20 and np.array_equal(back["pos"], part["pos"])
    rest = mdrun.advance(back, 20, chunk=20, checkpoint=path)
    assert rest["step"] == 40
    assert np.array_equal(rest["pos"], whole["pos"])
    assert np.array_equal(rest["vel"], whole["vel"])
    assert whole["log"].shape == (41, 6)
    assert np.array_equal(rest["log"], whole["log"])
    assert np.abs(whole["vel"]).max() > 0          # the ions did move
