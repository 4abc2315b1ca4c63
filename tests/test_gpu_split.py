"""A frame split by directions: plans built over slices of the direction grid
(what each rank of paper_2511_09165_b300.split runs) give the rows of the plan
over the whole grid.  One GPU runs every slice here; the exchange between
ranks is covered by tests/test_split_cpu.py."""
import numpy as np
import pytest

from workloads import scenes
from paper_2511_09165_b300.split import direction_slices, slice_grid

torch = pytest.importorskip("torch")
dm = pytest.importorskip("paper_2511_09165_b300")

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("mode", ["round", "linear"])
@pytest.mark.parametrize("world", [2, 3])
def test_slices_reassemble_the_whole_frame(mode, world):
    sc = scenes.hemi_3d(seed=2, n_samples=2048, n_dirs=600)
    dmode = dm.LINEAR if mode == "linear" else dm.ROUND
    kw = dict(mic_xyz=sc.mic_xyz, n_samples=sc.n_samples, fs=sc.fs, c=sc.c, order=5,
              delay_mode=dmode)
    x = torch.from_numpy(sc.frame).cuda()
    full_plan = dm.Plan(dir_unit=sc.dir_unit, **kw)
    full = full_plan(x).cpu().numpy()
    full_plan.check()
    full_plan.close()
    out = np.empty_like(full)
    for lo, hi in direction_slices(sc.n_dirs, world):
        _, unit, _ = slice_grid(dir_unit=sc.dir_unit, lo=lo, hi=hi)
        p = dm.Plan(dir_unit=unit, **kw)
        out[lo:hi] = p(x).cpu().numpy()
        p.check()
        p.close()
    assert np.array_equal(out, full)
