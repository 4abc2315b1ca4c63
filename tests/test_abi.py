"""The C-ABI library builds, loads and exports every symbol include/dmas.h
declares; host-side validation rejects bad arguments without a GPU."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

import paper_2511_09165_b300 as dm
from paper_2511_09165_b300 import build as dm_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    inc = os.path.join(ROOT, "include")
    for fn in os.listdir(inc):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(inc, fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(dmas_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    dm_build.build()
    return dm.load_library()


def test_exports_every_declared_symbol(lib):
    decl = declared_symbols()
    assert decl, "no declarations found"
    for name in sorted(decl):
        assert hasattr(lib, name), name
    assert decl == set(dm.EXPORTS)


def test_checked_build_exports_the_same_symbols():
    """The host-checked variant (DMAS_CHECKED) links and exports the same ABI."""
    path = dm_build.build(checked=True)
    chk = ctypes.CDLL(path)
    for name in sorted(declared_symbols()):
        assert hasattr(chk, name), name
    chk.dmas_status_string.restype = ctypes.c_char_p
    assert b"host-checked" in chk.dmas_status_string(6)


def test_status_strings_and_version(lib):
    for code in range(7):
        assert lib.dmas_status_string(code)
    assert lib.dmas_status_string(99) == b"unknown status"
    assert lib.dmas_version() >= 100


def _desc(**kw):
    xyz = np.zeros((4, 3))
    xyz[:, 0] = [0.0, 0.01, 0.02, 0.03]
    azel = np.zeros((3, 2))
    base = dict(n_mics=4, mic_xyz=xyz, n_dirs=3, dir_azel=azel, dir_unit=None, delays_s=None,
                n_samples=64, fs=450e3, c=343.0, order=5, delay_mode=0, flags=3, cf_eps=0.0,
                env_cutoff_hz=0.0, env_taps=0, chan_prec=0, ng_prec=0, mf_signal=None, mf_len=0)
    base.update(kw)
    keep = []

    def ptr(a):
        if a is None:
            return None
        a = np.ascontiguousarray(a, dtype=np.float64)
        keep.append(a)
        return a.ctypes.data_as(ctypes.c_void_p)

    d = dm.PlanDesc(base["n_mics"], ptr(base["mic_xyz"]), base["n_dirs"], ptr(base["dir_azel"]),
                    ptr(base["dir_unit"]), ptr(base["delays_s"]), base["n_samples"], base["fs"],
                    base["c"], base["order"], base["delay_mode"], base["flags"], base["cf_eps"],
                    base["env_cutoff_hz"], base["env_taps"], base["chan_prec"], base["ng_prec"],
                    None, base["mf_len"])
    if base["mf_signal"] is not None:
        e = np.ascontiguousarray(base["mf_signal"], dtype=np.float32)
        keep.append(e)
        d.mf_signal = e.ctypes.data_as(ctypes.c_void_p)
    return d, keep


BAD = [
    dict(n_mics=0), dict(n_mics=5000), dict(n_dirs=0), dict(n_samples=0),
    dict(n_samples=(1 << 24) + 1), dict(order=0), dict(order=9), dict(fs=0.0),
    dict(fs=math.nan), dict(fs=math.inf), dict(c=-1.0), dict(c=math.nan), dict(delay_mode=2),
    dict(chan_prec=3), dict(ng_prec=3), dict(flags=8), dict(mic_xyz=None),
    dict(dir_azel=None), dict(env_taps=2), dict(env_taps=1025), dict(env_cutoff_hz=300e3),
    dict(cf_eps=math.inf), dict(cf_eps=1e-60),
    dict(mic_xyz=np.full((4, 3), np.nan)),
    dict(delays_s=np.full((3, 4), np.inf)),
    dict(delays_s=np.full((3, 4), 10.0)),          # 4.5e6 samples of delay > 2^22
    dict(delays_s=np.array([[0.0] * 4, [0.1] * 4, [0.0] * 4])),  # group spread > shared memory
    dict(mf_signal=np.zeros(8193), mf_len=8193),   # emitted signal longer than 8192
    dict(mf_signal=None, mf_len=5),                 # length without a signal
    dict(mf_signal=np.ones(4), mf_len=0),           # signal without a length
    dict(mf_signal=np.array([1.0, np.nan]), mf_len=2),
    dict(mf_len=-1),
]


@pytest.mark.parametrize("kw", BAD)
def test_bad_descs_are_rejected_on_the_host(lib, kw):
    d, keep = _desc(**kw)
    h = ctypes.c_void_p()
    assert lib.dmas_plan_create(ctypes.byref(d), ctypes.byref(h)) == 1
    assert not h.value


def test_null_arguments(lib):
    h = ctypes.c_void_p()
    assert lib.dmas_plan_create(None, ctypes.byref(h)) == 1
    d, keep = _desc()
    assert lib.dmas_plan_create(ctypes.byref(d), None) == 1
    assert lib.dmas_destroy(None) == 0
    assert lib.dmas_beamform(None, None, None, None, None, None) == 1
    assert lib.dmas_beamform_host(None, None, None, None) == 1
    assert lib.dmas_beamform_batch(0, None, None, None, None, 0, None) == 1
    assert lib.dmas_batch_workspace_bytes(0, None) == 0
    assert lib.dmas_plan_workspace_bytes(None) == 0
    info = dm.PlanInfo()
    assert lib.dmas_plan_get_info(None, ctypes.byref(info)) == 1
    assert lib.dmas_plan_get_delays(None, None, None) == 1
    assert lib.dmas_plan_get_taps(None, None) == 1
    assert lib.dmas_plan_check(None) == 1
    assert lib.dmas_plan_last_error(None) == b""
    assert lib.dmas_plan_set_profiling(None, 1) == 1
    assert lib.dmas_plan_stage_ms(None, None, None, None) == 1
    assert lib.dmas_selftest_wait_timeout(0.0, None) == 1
    assert lib.dmas_selftest_wait_timeout(math.nan, None) == 1
    assert lib.dmas_beamform_noalloc(None, None, None, None) == 1


def test_python_binding_requires_geometry():
    with pytest.raises(ValueError):
        dm.Plan(n_samples=16, fs=1000.0)
