"""CPU checks of the CUDA library: it builds for sm_103a, loads, exports every
symbol the public headers declare, and rejects bad arguments on the host."""
import ctypes
import glob
import os
import re

import pytest

from paper_1909_00145_gb300 import scsc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(scsc_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


def test_headers_declare_the_boundary():
    names = declared_symbols()
    for need in ["scsc_create", "scsc_destroy", "scsc_code_step", "scsc_dict_step",
                 "scsc_objective", "scsc_mask", "scsc_synth", "scsc_synth_backward",
                 "scsc_lipschitz_codes", "scsc_last_error", "scsc_sync", "scsc_online_save",
                 "scsc_online_load", "scsc_online_reset", "scsc_online_state_size",
                 "scsc_code_step_host", "scsc_code_step_observed", "scsc_code_step_admm",
                 "scsc_objective_observed", "scsc_screen", "scsc_code_step_screened"]:
        assert need in names


def test_library_loads_and_exports_every_declared_symbol():
    L = scsc.lib()
    for name in declared_symbols():
        assert hasattr(L, name), name


def test_library_is_built_for_sm103a():
    path = scsc.library_path()
    data = open(path, "rb").read()
    assert b"sm_103a" in data or b"sm_103" in data


def test_config_validation_happens_on_the_host():
    L = scsc.lib()
    bad = [dict(K=0), dict(K=600), dict(s=4), dict(s=13), dict(lam=0.0), dict(p=(3, 2)),
           dict(p=(1, 0)), dict(step=-1.0), dict(flags=32), dict(prec=3)]
    for kw in bad:
        args = dict(K=16, s=11, lam=1.0, p=(1, 2), step=0.0, flags=0, prec=0)
        args.update(kw)
        cfg = scsc.scsc_config(args["K"], args["s"], args["lam"], args["p"][0], args["p"][1], 0,
                               args["prec"], args["step"], args["flags"])
        h = ctypes.c_void_p()
        assert L.scsc_create(ctypes.byref(cfg), None, ctypes.byref(h)) == scsc.SCSC_EINVAL, kw
        assert not h


def test_null_context_is_rejected():
    L = scsc.lib()
    assert L.scsc_destroy(None) == scsc.SCSC_OK
    assert L.scsc_sync(None) == scsc.SCSC_EINVAL
    assert L.scsc_code_step(None, None, None, None, None, 0, 1) == scsc.SCSC_EINVAL
    assert L.scsc_code_step_host(None, None, None, None, None, 0, 1) == scsc.SCSC_EINVAL
    assert L.scsc_code_step_observed(None, None, None, None, None, None, 0, 1) == scsc.SCSC_EINVAL
    assert L.scsc_code_step_admm(None, None, None, None, None, 0, 1, 1, 0.0, 0.0) == \
        scsc.SCSC_EINVAL
    assert L.scsc_screen(None, None, None, None, None, None, None, None) == scsc.SCSC_EINVAL
    assert L.scsc_code_step_screened(None, None, None, None, None, 0, 1, 1, None, None) == \
        scsc.SCSC_EINVAL


def test_batch_descriptor_layout():
    b = scsc.Batch([3, 5], [4, 2], ids=[7, 9])
    assert list(b.offsets) == [0, 12]
    assert b.total_pixels == 22
    assert ctypes.sizeof(scsc.scsc_config) == 56


def test_binding_checks_buffer_sizes_before_any_launch():
    torch = pytest.importorskip("torch")

    class Ctx:
        K, s = 20, 5

    b = scsc.Batch([3, 5], [4, 2])  # 22 pixels
    ok = dict(x=torch.zeros(22), d=torch.zeros(20 * 25), z=torch.zeros(22 * 20),
              observed=torch.zeros(22, dtype=torch.uint8), bits=torch.zeros(22, dtype=torch.int32))
    scsc._need_step(Ctx, b, **ok)
    scsc._need_step(Ctx, b, x=torch.zeros(40))  # larger is fine
    for name, bad in [("x", torch.zeros(21)), ("d", torch.zeros(20 * 25 - 1)),
                      ("z", torch.zeros(22 * 20 - 1)), ("observed", torch.zeros(22)),
                      ("bits", torch.zeros(21, dtype=torch.int32)),
                      ("x", torch.zeros(22, dtype=torch.float64))]:
        with pytest.raises(ValueError, match=name):
            scsc._need_step(Ctx, b, **{name: bad})


def test_objective_noalloc_binding_checks_buffers_before_any_launch():
    # short or wrongly typed buffers are rejected by the binding before the
    # library is called (CPU tensors: nothing could be launched on them)
    torch = pytest.importorskip("torch")
    K, s, n, H, W = 4, 3, 2, 8, 8
    P = n * H * W
    x = torch.zeros(P)
    z = torch.zeros(P * K)
    d = torch.zeros(K * s * s)
    out = torch.zeros(1, dtype=torch.float64)
    bad = [
        dict(z=torch.zeros(P)),                          # n H W values instead of n H W K
        dict(x=torch.zeros(P, dtype=torch.float64)),     # float64 image
        dict(z=torch.zeros(P * K, dtype=torch.float64)),
        dict(d=torch.zeros(K * s * s - 1)),
        dict(out=torch.zeros(1, dtype=torch.float32)),   # the result is one double
        dict(x=torch.zeros(P, dtype=torch.int32)),       # right size, not a float
        dict(x=None),
    ]
    for kw in bad:
        args = dict(x=x, z=z, d=d, out=out)
        args.update(kw)
        with pytest.raises(ValueError):
            scsc.scsc_objective_noalloc(K, s, 1.0, n, H, W, args["x"], args["z"], args["d"],
                                        args["out"])


def test_tf32_is_declared_and_reported_unsupported_on_the_host():
    """SCSC_TF32 is part of the precision enum; scsc_create rejects it with
    SCSC_EUNSUPPORTED (not EINVAL) before touching the device."""
    L = scsc.lib()
    cfg = scsc.scsc_config(16, 11, 1.0, 1, 2, 0, scsc.SCSC_TF32, 0.0, 0)
    h = ctypes.c_void_p()
    assert L.scsc_create(ctypes.byref(cfg), None, ctypes.byref(h)) == scsc.SCSC_EUNSUPPORTED
    assert not h
    text = open(os.path.join(ROOT, "include", "scsc.h")).read()
    assert "SCSC_TF32 = 2" in text and "SCSC_ENONFINITE = 5" in text
    assert "SCSC_FLAG_UNSAMPLED_KEEP 8u" in text
