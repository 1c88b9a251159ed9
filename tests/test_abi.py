"""The C-ABI library builds for sm_103a, loads, and exports every symbol include/art.h declares.
Host-only entry points are exercised; nothing here launches a kernel."""
import ctypes
import os
import re

import pytest

from paper_2103_07417_gb300 import art
from paper_2103_07417_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(art_[a-z0-9_]+)\s*\(", src))
    return names


def test_header_declarations_are_exported():
    lib = art.load()
    declared = _declared()
    assert {"art_create", "art_render", "art_trace_pixels", "art_refine_level"} <= declared
    for name in declared:
        assert hasattr(lib, name), name
    assert set(art.EXPORTS) <= declared


def test_image_size_and_planes_host_only():
    job = art.make_job(**W.cfg0())
    assert art.art_image_size(job) == (129, 129)
    assert art.art_planes(job) == 1
    job2 = art.make_job(**W.job(n0x=65, n0y=33, levels=4, subrings=3))
    assert art.art_image_size(job2) == (1025, 513)
    assert art.art_planes(job2) == 3
    bad = art.make_job(**W.job(n0x=1))
    with pytest.raises(RuntimeError):
        art.art_image_size(bad)


def test_strerror_names_codes():
    assert art.art_strerror(0) == "ok"
    assert "invalid" in art.art_strerror(art.ART_ERR_ARG)


def test_no_device_fails_loudly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    ctx = ctypes.c_void_p()
    rc = art.load().art_create(ctypes.byref(ctx), 0, None)
    assert rc == art.ART_ERR_CUDA
    with pytest.raises(RuntimeError):
        art.Context(0)
