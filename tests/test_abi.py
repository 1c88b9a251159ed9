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
    job = art.make_job(**W.schwarzschild_129())
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


def _struct_fields(name):
    src = open(os.path.join(ROOT, "include", "art.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    body = re.search(r"typedef struct %s \{(.*?)\} %s;" % (name, name), src, flags=re.S).group(1)
    out = []
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl:
            continue
        ctype, rest = decl.split(None, 1)
        for nm in rest.split(","):
            out.append((ctype, nm.strip().lstrip("*")))
    return out


def test_job_struct_matches_header():
    """The binding's art_job mirrors the header field by field (names, order, widths)."""
    fields = _struct_fields("art_job")
    width = {"double": ctypes.c_double, "int32_t": ctypes.c_int32}
    assert [n for _, n in fields] == [n for n, _ in art.Job._fields_]
    for (ctype, n), (pn, pt) in zip(fields, art.Job._fields_):
        assert width[ctype] == pt, n


def test_stats_struct_matches_header():
    """art_stats in the binding has the header's fields, in order, with the same sizes."""
    fields = _struct_fields("art_stats")
    names = [n for n, _ in art.Stats._fields_]
    assert names == [f[1].split("[")[0] for f in fields]
    assert ctypes.sizeof(art.Stats) == 8 * (len(fields) + 15)  # rays_per_level holds 16


def test_noalloc_rejects_grid_jobs_before_gpu_work():
    """A grid job has no context to hold its grid: the allocation-free call refuses it before
    touching any device state (checked on the host: an empty ray list, null pointers)."""
    job = art.make_job(**W.grmhd_8193(n0x=9, n0y=9, levels=0))
    rc = art.load().art_trace_pixels_noalloc(ctypes.byref(job), None, 0, None, None, None)
    assert rc == art.ART_ERR_UNSUPPORTED
