"""The allocation-free classification entry point (ebr_classify_cells_static).

It serves callers that cannot let the library allocate device memory (their
own memory pool or budget, or no cudaMalloc while other work runs).  It is
called here through the C ABI on buffers the test owns, twice in a row, and
its fluid / solid tags and interface count must equal those of the planned
path (ebr_plan): tags bit for bit, counts exactly.  On the small cases the
tags are also compared with the oracle's solid set and the count with a
brute-force count over the oracle's tags.  One case has exactly
EBR_STATIC_MAX_ROWS rows, where the last row run sits next to the status word
of the fixed array.  The file sorts last so a run that stops at the first
failure has already run every other test."""

import ctypes

import numpy as np
import pytest
import torch

from paper_2609_10165_b300 import _lib
from paper_2609_10165_b300 import inputs as I
from paper_2609_10165_b300.api import Reconstructor, _grid_struct, _body_struct

pytestmark = pytest.mark.gpu

MAX_ROWS = 1 << 18                         # EBR_STATIC_MAX_ROWS

CASES = {
    # n_y n_z == EBR_STATIC_MAX_ROWS exactly
    "max_rows_sphere": lambda: {"grid": I.grid(3, [8, 512, 512], [-1.0] * 3, [1.0] * 3),
                                "body": I.sphere(0.013, -0.007, 0.011, 0.6)},
    "cylinder_128": lambda: I.cylinder(128, 1),
    "airfoil_2048": lambda: I.airfoil_2048(),
    "sphere_256": lambda: I.sphere_cfg(256, 5),
    "batch_geometry_7": lambda: I.batch()[7],
    "ragged_ellipse": lambda: {"grid": I.grid(2, [37, 29], [-1.0, -1.0], [1.0, 1.0]),
                               "body": I.ellipse(0.03, -0.02, 0.6, 0.35, 0.7)},
}


def _call(lib, g, b, tags, count):
    gs = _grid_struct(g)
    bs = _body_struct(b)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.ebr_classify_cells_static(ctypes.byref(gs), ctypes.byref(bs),
                                         ctypes.c_void_p(tags.data_ptr()),
                                         ctypes.c_void_p(count.data_ptr()), stream)


ORACLE_CASES = ("cylinder_128", "ragged_ellipse", "batch_geometry_7")


def _oracle_solid_and_count(g, b):
    """Solid set (centre in the closed body) and brute-force interface count
    (cells with a face neighbour on the other side) from the oracle."""
    import oracle as O
    c = O.classify(g, b, "HGC")
    solid = ((c.tags == 1) | (c.tags == 2)).astype(np.int8)
    n = [int(v) for v in g["n"]][: g["dim"]]
    sv = solid.reshape(n[::-1])                 # [.., y, x]: x fastest
    iface = np.zeros(sv.shape, bool)
    for ax in range(sv.ndim):
        diff = np.diff(sv, axis=ax) != 0
        lo = [slice(None)] * sv.ndim
        hi = [slice(None)] * sv.ndim
        lo[ax] = slice(0, -1)
        hi[ax] = slice(1, None)
        iface[tuple(lo)] |= diff
        iface[tuple(hi)] |= diff
    return solid, int(iface.sum())


@pytest.mark.parametrize("name", sorted(CASES))
def test_static_entry_point_matches_planned_path(name):
    lib = _lib.load()
    w = CASES[name]()
    g, b = w["grid"], w["body"]
    R = Reconstructor(g, b, "HGC")
    ref_tags = R.tags.cpu().numpy()
    ref_solid = ((ref_tags == 1) | (ref_tags == 2)).astype(np.int8)
    ref_count = R.counts()[0]["n_interface"]
    n = R.n_cells
    if name in ORACLE_CASES:
        o_solid, o_count = _oracle_solid_and_count(g, b)
        assert np.array_equal(o_solid, ref_solid) and o_count == ref_count, name
    if name == "max_rows_sphere":
        assert g["n"][1] * g["n"][2] == MAX_ROWS
    for call in range(2):
        tags = torch.full((n,), 7, dtype=torch.int8, device="cuda")
        count = torch.full((1,), -5, dtype=torch.int64, device="cuda")
        assert _call(lib, g, b, tags, count) == 0
        torch.cuda.synchronize()
        assert np.array_equal(tags.cpu().numpy(), ref_solid), (name, call)
        assert int(count.item()) == ref_count, (name, call, int(count.item()), ref_count)


def test_static_entry_point_rejects_too_many_rows():
    lib = _lib.load()
    rows = (1 << 18) + 4                       # n_y * n_z above the fixed scratch
    g = I.grid(3, [4, 1024, rows // 1024 + 1], [-1.0] * 3, [1.0] * 3)
    b = I.sphere(0.0, 0.0, 0.0, 0.5)
    tags = torch.zeros(16, dtype=torch.int8, device="cuda")
    count = torch.zeros(1, dtype=torch.int64, device="cuda")
    assert _call(lib, g, b, tags, count) == -1          # EBR_EINVAL, nothing launched
    torch.cuda.synchronize()
    assert int(count.item()) == 0
