"""Batched launches and the continuous-batching server.

A frame's image must not depend on the batch it runs in: every entry has its
own scratch and the per-pixel arithmetic is the same, so the comparison with
dmas_beamform of the frame alone is bitwise.
"""
import functools
import gc
import time

import numpy as np
import pytest

from workloads import scenes

torch = pytest.importorskip("torch")
dm = pytest.importorskip("paper_2511_09165_b300")
from paper_2511_09165_b300 import serving  # noqa: E402

pytestmark = pytest.mark.gpu


def _plan(sc, order, mode, **kw):
    return dm.Plan(mic_xyz=sc.mic_xyz, dir_azel=sc.dir_azel, dir_unit=sc.dir_unit,
                   n_samples=sc.n_samples, fs=sc.fs, c=sc.c, order=order, delay_mode=mode, **kw)


def test_batch_of_mixed_variants_is_bitwise_equal_to_single_calls():
    a = scenes.small_2d(seed=1, n_samples=1500)
    b = scenes.hemi_3d(seed=2, n_samples=1100, n_dirs=100)
    c = scenes.passive(seed=4, n_mics=40, n_samples=900, n_az=12, n_el=6)
    # large enough for the tensor-core envelope (more than 1.5e8 tap products)
    d = scenes.hemi_3d(seed=2, n_samples=4100, n_dirs=1200)
    plans = [
        _plan(a, 5, dm.ROUND), _plan(a, 3, dm.ROUND), _plan(b, 5, dm.LINEAR),
        _plan(b, 2, dm.LINEAR, ng_prec=dm.NG_CF32), _plan(a, 7, dm.ROUND),
        _plan(a, 5, dm.ROUND, chan_prec=dm.CH_F16), _plan(c, 4, dm.ROUND, envelope=False),
        _plan(a, 5, dm.ROUND, env_taps=51), _plan(c, 5, dm.LINEAR, cf=False),
        _plan(d, 3, dm.LINEAR), _plan(d, 5, dm.ROUND),
    ]
    scs = [a, a, b, b, a, a, c, a, c, d, d]
    frames = [torch.from_numpy(sc.frame).cuda() for sc in scs]
    alone = [p(f).clone() for p, f in zip(plans, frames)]
    # every plan twice, interleaved, in one batch
    order = list(range(len(plans))) * 2
    imgs = dm.beamform_batch([plans[k] for k in order], [frames[k] for k in order])
    torch.cuda.synchronize()
    for k, im in zip(order, imgs):
        assert torch.equal(im, alone[k]), k
    # the same batch from host frames in one call (upload, batch, completion event)
    bp = [plans[k] for k in order]
    hosts = [torch.from_numpy(scs[k].frame).pin_memory() for k in order]
    dev = [torch.empty((p.n_mics, p.n_samples), device="cuda") for p in bp]
    out = [torch.empty((p.n_dirs, p.n_samples), device="cuda") for p in bp]
    ws = torch.empty(dm.batch_workspace_bytes(bp), device="cuda", dtype=torch.uint8)
    done = torch.cuda.Event()
    done.record()                           # the event exists before the call records it
    dm.beamform_batch_upload(bp, hosts, dev, out, ws, done_event=done)
    done.synchronize()
    for k, im in zip(order, out):
        assert torch.equal(im, alone[k]), k
    for p in plans:
        p.check()
        p.close()


@functools.lru_cache(maxsize=None)
def _small_mix():
    return scenes.serving_mix(seed=7, n_sensors=6, frames_per_sensor=2, mics=(32, 48),
                              dirs=(91, 2048), samples=(2048, 4096), orders=(3, 5))


def _sensors(mix):
    out = []
    for s in mix:
        plan = dm.Plan(mic_xyz=s.mic_xyz, dir_azel=s.dir_azel, dir_unit=s.dir_unit,
                       n_samples=s.n_samples, fs=s.fs, c=s.c, order=s.order)
        out.append(serving.Sensor(plan, s.name))
    return out


def test_server_results_equal_alone_and_in_the_mix():
    mix = _small_mix()
    sensors = _sensors(mix)
    host = [[torch.from_numpy(f).pin_memory() for f in s.frames] for s in mix]
    rng = np.random.default_rng(3)
    reqs = []
    with serving.Server(sensors, streams=2, max_batch=16) as srv:
        for k in range(48):
            si = int(rng.integers(len(mix)))
            fi = int(rng.integers(len(host[si])))
            reqs.append((si, fi, srv.submit(si, host[si][fi], keep_image=True)))
            if k % 12 == 11:
                time.sleep(0.002)           # arrivals while batches run
        assert srv.drain(120.0)
        assert srv.batches < len(reqs)      # frames were batched together
    assert max(r.batch_size for _, _, r in reqs) > 1
    for si, fi, r in reqs:
        assert not r.rejected and r.latency > 0
        alone = sensors[si].plan(host[si][fi].cuda())
        assert torch.equal(r.image, alone)
    for s in sensors:
        s.plan.close()


def test_server_admission_by_memory_and_rejection():
    mix = _small_mix()
    sensors = _sensors(mix)
    sizes = [s.device_bytes for s in sensors]
    budget = max(sizes)                     # one frame of the largest sensor at a time
    host = [torch.from_numpy(s.frames[0]).pin_memory() for s in mix]
    with serving.Server(sensors, budget_bytes=budget, streams=2) as srv:
        reqs = [srv.submit(k % len(mix), host[k % len(mix)], keep_image=True) for k in range(12)]
        assert srv.drain(120.0)
    assert all(not r.rejected for r in reqs)
    for k, r in enumerate(reqs):
        assert torch.equal(r.image, sensors[k % len(mix)].plan(host[k % len(mix)].cuda()))
    small = serving.Server(sensors, budget_bytes=min(sizes) - 1, streams=1)
    with small:
        r = small.submit(0, host[0])
        assert small.drain(30.0)
    assert r.rejected
    for s in sensors:
        s.plan.close()


def test_handed_over_image_lives_as_long_as_its_tensor():
    """The server hands device images over through the CUDA array interface;
    torch keeps the holder (whose finaliser frees the image) alive for as long
    as a tensor over it exists."""
    class Holder:
        freed = False

        def __init__(self, t):
            self.t = t
            self.__cuda_array_interface__ = t.__cuda_array_interface__

        def __del__(self):
            Holder.freed = True

    h = Holder(torch.zeros(4, device="cuda"))
    x = torch.as_tensor(h, device="cuda")
    del h
    gc.collect()
    assert not Holder.freed
    del x
    gc.collect()
    assert Holder.freed


def test_server_images_outlive_the_server():
    mix = _small_mix()
    sensors = _sensors(mix)
    host = [torch.from_numpy(s.frames[0]).pin_memory() for s in mix]
    with serving.Server(sensors, streams=2) as srv:
        reqs = [srv.submit(k, host[k], keep_image=True) for k in range(len(mix))]
        assert srv.drain(60.0)
    images = [r.image for r in reqs]
    del reqs, srv
    gc.collect()
    for k, im in enumerate(images):
        assert torch.equal(im, sensors[k].plan(host[k].cuda()))
    for s in sensors:
        s.plan.close()


def test_one_frame_per_launch_baseline_matches():
    mix = _small_mix()
    sensors = _sensors(mix)
    host = [torch.from_numpy(s.frames[0]).pin_memory() for s in mix]
    t0 = time.perf_counter()
    reqs = [serving.Request(k, host[k], t0 + 0.001 * k, keep_image=True) for k in range(len(mix))]
    serving.one_frame_per_launch(sensors, reqs)
    for k, r in enumerate(reqs):
        assert r.t_done >= r.t_arrival
        assert torch.equal(r.image, sensors[k].plan(host[k].cuda()))
    for s in sensors:
        s.plan.close()


def test_frame_path_replays_from_a_cuda_graph():
    """dmas_beamform only enqueues kernels on its stream (no allocation, no
    synchronisation), so it can be captured into a CUDA graph; a replay on a
    new frame written into the captured input gives the direct call's image
    bit for bit."""
    sc = scenes.small_2d(seed=1)
    plan = dm.Plan(mic_xyz=sc.mic_xyz, dir_azel=sc.dir_azel, n_samples=sc.n_samples, fs=sc.fs,
                   c=sc.c, order=5, delay_mode=dm.ROUND)
    frame = torch.from_numpy(sc.frame).cuda()
    image = torch.empty((sc.n_dirs, sc.n_samples), device="cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        plan(frame, out=image, stream=s)          # warm-up outside the capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        plan(frame, out=image, stream=s)
    other = scenes.small_2d(seed=3)
    frame.copy_(torch.from_numpy(other.frame))
    g.replay()
    torch.cuda.synchronize()
    plan.check()
    ref = plan(torch.from_numpy(other.frame).cuda())
    torch.cuda.synchronize()
    assert torch.equal(image, ref)
    plan.close()


@pytest.mark.parametrize("cap", [1, 3, 16])
def test_envelope_tile_cap_changes_scheduling_not_results(cap):
    """dmas_plan_set_envelope_tile_cap retires the tensor-core envelope's CTAs
    every `cap` tiles; the image is bitwise the uncapped one, alone and in a
    batch."""
    sc = scenes.hemi_3d(seed=2, n_samples=4100, n_dirs=1200)   # tensor-core envelope
    plan = _plan(sc, 5, dm.LINEAR)
    x = torch.from_numpy(sc.frame).cuda()
    want = plan(x).clone()
    plan.set_envelope_tile_cap(cap)
    got = plan(x).clone()
    b1, b2 = dm.beamform_batch([plan, plan], [x, x])
    plan.set_envelope_tile_cap(0)
    again = plan(x)
    torch.cuda.synchronize()
    plan.check()
    plan.close()
    assert torch.equal(got, want) and torch.equal(b1, want) and torch.equal(b2, want)
    assert torch.equal(again, want)
