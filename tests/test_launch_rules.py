"""Source rules of the kernel launches (read as text; no GPU).

A kernel launched through the library's launch() helper may be scheduled
before the kernel ahead of it in the stream has finished (programmatic
dependent launch), so its body must begin with pdl_enter(), which waits for
the preceding grids before any memory is touched.  Every launch site is
checked against the kernel's definition."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2609_10165_b300", "csrc")


def _sources():
    out = {}
    for fn in sorted(os.listdir(CSRC)):
        if fn.endswith((".cu", ".cuh")):
            with open(os.path.join(CSRC, fn)) as f:
                out[fn] = f.read()
    return out


def _launched(srcs):
    names = set()
    for s in srcs.values():
        for m in re.finditer(r"\blaunch\(\s*(k_[A-Za-z0-9_]+)", s):
            names.add(m.group(1))
    return names


def _bodies(srcs, name):
    """Opening of the body of every __global__ definition of `name`."""
    out = []
    for fn, s in srcs.items():
        for m in re.finditer(r"__global__[^;{]*?\b" + re.escape(name) + r"\s*\(", s):
            d, i = 0, m.end() - 1
            while True:
                if s[i] == "(":
                    d += 1
                elif s[i] == ")":
                    d -= 1
                    if d == 0:
                        break
                i += 1
            b = s.index("{", i)
            out.append((fn, s[b + 1:b + 200]))
    return out


def test_every_launched_kernel_waits_first():
    srcs = _sources()
    names = _launched(srcs)
    assert len(names) > 30
    for name in sorted(names):
        bodies = _bodies(srcs, name)
        assert bodies, "no definition of %s" % name
        for fn, body in bodies:
            first = body.lstrip().split(";", 1)[0]
            assert first == "pdl_enter()", "%s in %s: first statement %r" % (name, fn, first)


def test_no_plain_launch_of_a_kernel_that_waits_is_needed():
    # kernels launched with <<< >>> are plain launches (full stream order);
    # they are the cooperative tiled fill, the allocation-free entry point's
    # kernels and the statistics
    srcs = _sources()
    plain = set()
    for s in srcs.values():
        for m in re.finditer(r"\b(k_[A-Za-z0-9_]+)(<[^<>]*>)?<<<", s):
            plain.add(m.group(1))
    assert plain <= {"k_rows_static", "k_iface_count_static", "k_static_status", "k_stats"}, plain


def test_pdl_switch_round_trip():
    from paper_2609_10165_b300 import _lib, build
    if not os.path.exists(_lib.LIB_PATH):
        build.build()
    lib = _lib.load()
    assert lib.ebr_get_pdl() == 1
    lib.ebr_set_pdl(0)
    try:
        assert lib.ebr_get_pdl() == 0
    finally:
        lib.ebr_set_pdl(1)
    assert lib.ebr_get_pdl() == 1
