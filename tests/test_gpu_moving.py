"""Moving bodies (Sec. 7): a geometry set whose bodies translate and rotate
is advanced step by step through ebr_move + ebr_build_levels + fill +
forces + adjoint (paper_2609_10165_b300.moving).  At every step the tags,
ghost lists, levels and r_i equal the oracle's for the moved bodies bit for
bit, psi / n / S agree with the oracle's closest points, the ghost values
and forces match the oracle (FP32 tolerances) and the gradient matches the
oracle's; once the capacity has settled the steps allocate no device
memory."""

import numpy as np
import pytest
import torch

import oracle as O
from paper_2609_10165_b300 import inputs as I
from paper_2609_10165_b300.moving import MovingStepper, RigidMotion
from tests.parity import compare_geometry, oracle_bcs

pytestmark = pytest.mark.gpu


def _setup(dtype=torch.float32):
    grids = [I.grid(2, [96, 80], [-1.0, -1.0], [1.0, 1.0]),
             I.grid(2, [150, 70], [-1.0, -1.0], [3.0, 1.0]),
             I.grid(2, [64, 64], [-1.0, -1.0], [1.0, 1.0])]
    motions = [RigidMotion(I.ellipse(0.02, -0.03, 0.55, 0.3, 0.4), velocity=(0.05, -0.03, 0.0), omega=0.7),
               RigidMotion(I.airfoil(0.0, 0.0, 0.12, 1.0, 5.0), velocity=(0.02, 0.01, 0.0), omega=0.06),
               RigidMotion(I.circle(0.01, 0.02, 0.45), velocity=(0.1, 0.05, 0.0))]
    fields = [[I.FourierField(2, 4, g["lo"], g["hi"], 2100 + 10 * b + f) for b, g in enumerate(grids)]
              for f in range(3)]
    st = MovingStepper(grids, motions, fields, [I.DIRICHLET, I.DIRICHLET, I.NEUMANN], [0, 1], 2, 0.01,
                       I.DRAG_LIFT_DIRS_2D, dtype=dtype)
    return st, grids, motions, fields


def test_moving_bodies_match_the_oracle_every_step():
    st, grids, motions, fields = _setup()
    R = st.R
    allocs = []
    for step in range(12):
        forces, info, bcs, gf, gb = st.advance(0.05, adjoint=True)
        R.sync_status()
        allocs.append(R.diagnostics()["allocations"])
        if step % 3 != 0 and step < 11:
            continue
        tags = R.tags.cpu().numpy()
        work = [w.double().cpu().numpy() for w in st.work]
        fo = forces.cpu().numpy()
        gfh = [t.double().cpu().numpy() for t in gf]
        gbh = [t.double().cpu().numpy() for t in gb]
        for b, g in enumerate(grids):
            body = motions[b].at(st.t)
            o0, o1 = R.cell_offset[b], R.cell_offset[b + 1]
            c = O.classify(g, body, "HGC")
            assert c.ties == []
            lev = O.build_levels(c)
            assert np.array_equal(tags[o0:o1], c.tags), (step, b)
            sel = info["geom"] == b
            assert np.array_equal(info["cell"][sel], c.idx[lev.order]), (step, b)
            assert np.array_equal(info["level"][sel], lev.level[lev.order]), (step, b)
            compare_geometry(info["psi"][sel], info["normal"][sel], info["S"][sel], c, lev, tag=(step, b))
            # the oracle on the same field values (FP32, the previous ghost
            # cells restored) with boundary data at its own S
            arrays = [np.asarray(p.cpu().numpy()[o0:o1], dtype=np.float64) for p in st.pristine]
            wl = {"fields": [f[b] for f in fields], "bc": st.kinds}
            filled = O.fill(c, lev, arrays, st.kinds, oracle_bcs(wl, c, lev, f32=True))
            cells = c.idx[lev.order]
            for f in range(3):
                assert np.max(np.abs(work[f][o0:o1][cells] - filled[f][cells])) <= 1e-5 * np.abs(arrays[f]).max()
            ref, scale = O.forces(c, lev, filled[2], [filled[0], filled[1]], st.mu, st.dirs)
            assert np.all(np.abs(fo[b] - ref) <= 1e-4 * scale), (step, b, fo[b], ref)
            gx, gbo = O.adjoint_gradient(c, lev, st.kinds, 2, [0, 1], st.mu, st.dirs, (1.0, 1.0))
            for f in range(3):
                sc = max(np.abs(gx[f]).max(), np.abs(gbo[f]).max(), 1e-300)
                assert np.max(np.abs(gfh[f][o0:o1] - gx[f])) <= 2e-5 * sc, (step, b, f)
                assert np.max(np.abs(gbh[f][sel] - gbo[f])) <= 2e-5 * sc, (step, b, f)
    # the capacity settles: the last steps allocate nothing
    assert allocs[-1] == allocs[-6], allocs


def test_invalid_move_changes_nothing():
    from paper_2609_10165_b300._lib import EBRError
    st, grids, motions, fields = _setup()
    R = st.R
    info0 = R.ghost_info()
    bad = [motions[0].at(0.0), I.circle(0.0, 0.0, -1.0), motions[2].at(0.0)]
    with pytest.raises(EBRError) as ei:
        R.move(bad)
    assert ei.value.name == "EBR_EINVAL"
    # the plan is intact: the levels, fill and the next move work
    st.advance(0.05)
    R.sync_status()
    assert R.ghost_info()["cell"].size > 0 and info0["cell"].size > 0
