"""A frame split by directions across ranks (paper_2511_09165_b300.split):
the slicing, and the broadcast of the frame and gather of the rows with two and
three gloo ranks on the CPU, each rank's rows computed by the oracle for its
slice, compared with the oracle over the whole grid."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

from paper_2511_09165_b300.split import direction_slices, slice_grid  # noqa: E402


def test_slices_cover_the_grid_in_whole_groups():
    for n, w in [(2048, 2), (2048, 8), (91, 2), (91, 4), (8192, 3), (5, 4), (0, 2), (17, 1)]:
        s = direction_slices(n, w)
        assert len(s) == w
        assert s[0][0] == 0 and s[-1][1] == n
        for (a, b), (c, d) in zip(s, s[1:]):
            assert b == c and a <= b
        for lo, hi in s[:-1]:
            assert lo % 8 == 0 and hi % 8 == 0
        sizes = [hi - lo for lo, hi in s]
        assert max(sizes) - min(sizes) <= 8 or n < 8 * w


def test_slice_grid_cuts_whichever_description_is_given():
    az = np.arange(20.0).reshape(10, 2)
    a, u, d = slice_grid(dir_azel=az, lo=3, hi=7)
    assert u is None and d is None and np.array_equal(a, az[3:7])


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    import torch.distributed as td
    import oracle
    from paper_2511_09165_b300.split import SplitBeamformer
    from workloads import scenes
    td.init_process_group("gloo", rank=rank, world_size=world)
    sc = scenes.small_2d(seed=1, n_samples=600)
    u = oracle.unit_vectors(sc.dir_azel)
    tau = oracle.geometric_delays(sc.mic_xyz, u, sc.c)
    taps = oracle.fir_taps(sc.fs, 5000.0)

    def rows(frame, lo, hi):
        r = oracle.dmas(frame.numpy().astype(np.float64), tau, sc.fs, 3, oracle.LINEAR,
                        use_cf=True, taps=taps, dir_range=(lo, hi))
        return torch.from_numpy(r["img"].astype(np.float32))

    sb = SplitBeamformer(rank, world, sc.n_dirs, rows)
    # only the source rank holds the frame; the others start from zeros
    frame = torch.from_numpy(sc.frame) if rank == 0 else torch.zeros(sc.frame.shape)
    img = sb(frame, src=0, dst=0)
    if rank == 0:
        full = oracle.dmas(sc.frame.astype(np.float64), tau, sc.fs, 3, oracle.LINEAR,
                           use_cf=True, taps=taps)["img"].astype(np.float32)
        q.put(bool(np.array_equal(img.numpy(), full)))
    else:
        q.put(img is None)
    td.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_ranks_assemble_the_whole_image(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(300)
        assert p.exitcode == 0
    assert all(q.get(timeout=10) for _ in range(world))
