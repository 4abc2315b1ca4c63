"""dmas_beamform_noalloc: beamforming for callers that may allocate at set-up
but must not allocate device memory while processing frames (a real-time loop
with a frame deadline cannot afford a cudaMalloc, which may synchronise the
device and take an unbounded time).  Its scratch is a static device array
inside the library.

The tests call the entry point through the C ABI twice in a row, on two
different frames, and compare each result with dmas_beamform on the same plan
and frame: once with nearest-sample delays, once with interpolated delays
(whose kernel reads the root rows through a tensor map built over whichever
scratch the call uses, so alternating the two entry points on one plan must
rebuild it each time).  One more captures the call in a CUDA graph in global
capture mode, which fails if anything in the captured call allocates.  They
live in their own file, collected last, and pass both alone in a fresh process
and after the rest of the suite.
"""
import ctypes

import numpy as np
import pytest

from workloads import scenes
from parity import TOL_F32, eps_peak

torch = pytest.importorskip("torch")
dm = pytest.importorskip("paper_2511_09165_b300")

pytestmark = pytest.mark.gpu


def _call_noalloc(lib, plan, frame, image):
    stream = torch.cuda.current_stream().cuda_stream
    return lib.dmas_beamform_noalloc(plan.handle, ctypes.c_void_p(frame.data_ptr()),
                                     ctypes.c_void_p(image.data_ptr()),
                                     ctypes.c_void_p(stream))


def test_noalloc_matches_beamform_on_two_calls_in_a_row():
    lib = dm.load_library()
    sc = scenes.small_2d(seed=1)            # 32 mics, 91 azimuths, 4096 samples
    plan = dm.Plan(mic_xyz=sc.mic_xyz, dir_azel=sc.dir_azel, n_samples=sc.n_samples,
                   fs=sc.fs, c=sc.c, order=5, delay_mode=dm.ROUND)
    assert plan.workspace_bytes() <= 16 << 20
    frames = [torch.from_numpy(sc.frame).cuda(),
              torch.from_numpy(scenes.small_2d(seed=11).frame).cuda()]
    for frame in frames:
        want = plan(frame)
        got = torch.full_like(want, float("nan"))
        assert _call_noalloc(lib, plan, frame, got) == 0
        torch.cuda.synchronize()
        plan.check()
        w, g = want.cpu().numpy(), got.cpu().numpy()
        assert np.all(np.isfinite(g))
        assert eps_peak(g, w) <= TOL_F32
    plan.close()


def test_noalloc_interpolated_delays_alternating_with_beamform():
    lib = dm.load_library()
    sc = scenes.hemi_3d(seed=2, n_samples=2048, n_dirs=256)   # linear delays, 2 MiB y
    plan = dm.Plan(mic_xyz=sc.mic_xyz, dir_unit=sc.dir_unit, n_samples=sc.n_samples,
                   fs=sc.fs, c=sc.c, order=5, delay_mode=dm.LINEAR)
    assert plan.workspace_bytes() <= 16 << 20
    frames = [torch.from_numpy(sc.frame).cuda(),
              torch.from_numpy(scenes.hemi_3d(seed=12, n_samples=2048, n_dirs=256).frame).cuda()]
    for frame in frames:
        want = plan(frame).clone()                  # plan scratch
        got = torch.full_like(want, float("nan"))
        assert _call_noalloc(lib, plan, frame, got) == 0   # static scratch
        again = plan(frame)                         # plan scratch again
        torch.cuda.synchronize()
        plan.check()
        w, g, a = want.cpu().numpy(), got.cpu().numpy(), again.cpu().numpy()
        assert np.all(np.isfinite(g))
        assert eps_peak(g, w) <= TOL_F32
        assert np.array_equal(a, w)
    plan.close()


def test_noalloc_rejects_plans_larger_than_its_scratch():
    lib = dm.load_library()
    sc = scenes.hemi_3d(seed=2, n_samples=2048, n_dirs=2048)   # 16 MiB of pre-envelope image
    plan = dm.Plan(mic_xyz=sc.mic_xyz, dir_unit=sc.dir_unit, n_samples=sc.n_samples,
                   fs=sc.fs, c=sc.c, order=5, delay_mode=dm.LINEAR)
    assert plan.workspace_bytes() > 16 << 20
    frame = torch.from_numpy(sc.frame).cuda()
    image = torch.zeros((sc.n_dirs, sc.n_samples), device="cuda")
    assert _call_noalloc(lib, plan, frame, image) == 1       # DMAS_EINVAL
    msg = lib.dmas_plan_last_error(plan.handle).decode()
    assert "static" in msg and str(16 << 20) in msg
    assert torch.count_nonzero(image).item() == 0             # nothing was launched
    plan.close()


def test_noalloc_call_captures_in_a_global_mode_cuda_graph():
    """A CUDA graph captured in global mode fails if anything in the captured
    region allocates device memory, so a capture that succeeds shows that the
    call allocates nothing; the replayed graph must give the image of an
    ordinary call."""
    lib = dm.load_library()
    sc = scenes.hemi_3d(seed=4, n_samples=2048, n_dirs=256)   # linear delays
    plan = dm.Plan(mic_xyz=sc.mic_xyz, dir_unit=sc.dir_unit, n_samples=sc.n_samples,
                   fs=sc.fs, c=sc.c, order=5, delay_mode=dm.LINEAR)
    frame = torch.from_numpy(sc.frame).cuda()
    want = plan(frame).clone()
    got = torch.full_like(want, float("nan"))
    # one warm call: the static array's address and the tensor map over it are
    # looked up before the capture
    assert _call_noalloc(lib, plan, frame, got) == 0
    torch.cuda.synchronize()
    got.fill_(float("nan"))
    graph = torch.cuda.CUDAGraph()
    statuses = []
    with torch.cuda.graph(graph, capture_error_mode="global"):
        statuses.append(_call_noalloc(lib, plan, frame, got))
    assert statuses == [0]
    torch.cuda.synchronize()
    assert torch.isnan(got).all()           # capturing ran nothing
    graph.replay()
    torch.cuda.synchronize()
    plan.check()
    g, w = got.cpu().numpy(), want.cpu().numpy()
    assert np.all(np.isfinite(g))
    assert eps_peak(g, w) <= TOL_F32
    del graph
    plan.close()
