"""Python binding of the C ABI (include/ebr.h) for torch tensors.

PyTorch provides device memory and the current stream; every step of the
path runs in the library's CUDA kernels.  Geometry and body descriptions are
plain dicts (see ``inputs``): grid {"dim", "n", "lo", "hi"} and body
{"kind", "centre", "radii", "rot", "thickness", "chord"}.
"""

import ctypes

import numpy as np
import torch

from . import _lib

KIND = {"circle": 0, "sphere": 1, "ellipse": 2, "airfoil": 3}
PLACEMENT = {"HGC": 0, "CGC": 1, "CGC_ES": 2}
MODE = {"level": 0, "persistent": 1}
DTYPE = {torch.float32: 0, torch.float64: 1}
SECOND_LAYER = 16          # EBR_SECOND_LAYER


def _grid_struct(g):
    s = _lib.Grid()
    s.dim = int(g["dim"])
    n = list(g["n"]) + [1] * (3 - len(g["n"]))
    lo = list(g["lo"]) + [0.0] * (3 - len(g["lo"]))
    hi = list(g["hi"]) + [1.0] * (3 - len(g["hi"]))
    for a in range(3):
        s.n[a] = int(n[a]) if a < s.dim else 1
        s.lo[a] = float(lo[a]) if a < s.dim else 0.0
        s.hi[a] = float(hi[a]) if a < s.dim else 1.0
    return s


def _body_struct(b):
    s = _lib.Body()
    s.kind = KIND[b["kind"]]
    for a in range(3):
        s.centre[a] = float(b["centre"][a]) if a < len(b["centre"]) else 0.0
        s.radii[a] = float(b["radii"][a]) if a < len(b["radii"]) else 0.0
    for q in range(9):
        s.rot[q] = float(b["rot"][q])
    s.thickness = float(b.get("thickness", 0.0))
    s.chord = float(b.get("chord", 0.0))
    return s


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _ptr_array(ts):
    arr = (ctypes.c_void_p * len(ts))()
    for i, t in enumerate(ts):
        arr[i] = t.data_ptr() if t is not None else 0
    return arr


def set_pdl(enable):
    """Programmatic dependent launch of the library's kernels (process-wide,
    on by default): ebr_set_pdl."""
    _lib.load().ebr_set_pdl(1 if enable else 0)


def get_pdl():
    return bool(_lib.load().ebr_get_pdl())


class Reconstructor:
    """One planned geometry set (B >= 1 grids with bodies) on one device."""

    def __init__(self, grids, bodies, placement="HGC", device=None, layers=1):
        self.lib = _lib.load()
        if isinstance(grids, dict):
            grids, bodies = [grids], [bodies]
        self.B = len(grids)
        self.dim = int(grids[0]["dim"])
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.placement = placement
        h = ctypes.c_void_p()
        self._check(self.lib.ebr_create(ctypes.byref(h)), ctx=None)
        self.ctx = h
        self._grids = (_lib.Grid * self.B)(*[_grid_struct(g) for g in grids])
        self._bodies = (_lib.Body * self.B)(*[_body_struct(b) for b in bodies])
        ncell = sum(int(np.prod([g["n"][a] for a in range(int(g["dim"]))])) for g in grids)
        self.tags = torch.empty(ncell, dtype=torch.int8, device=self.device)
        if layers not in (1, 2):
            raise ValueError("layers must be 1 or 2")
        self.layers = layers
        flags = PLACEMENT[placement] | (SECOND_LAYER if layers == 2 else 0)
        if any("faces" in g for g in grids):
            # stretched grids: the faces of every axis, concatenated per geometry
            self._faces = [np.ascontiguousarray(np.concatenate([np.asarray(g["faces"][a], dtype=np.float64)
                                                                for a in range(int(g["dim"]))]))
                           if "faces" in g else None for g in grids]
            fp = (ctypes.c_void_p * self.B)(*[f.ctypes.data if f is not None else 0 for f in self._faces])
            self._check(self.lib.ebr_plan_faces(self.ctx, self.B, self._grids, fp, self._bodies,
                                                flags, _ptr(self.tags), self._stream()))
        else:
            self._check(self.lib.ebr_plan(self.ctx, self.B, self._grids, self._bodies,
                                          flags, _ptr(self.tags), self._stream()))
        off = (ctypes.c_int64 * (self.B + 1))()
        self._check(self.lib.ebr_layout(self.ctx, off))
        self.cell_offset = np.array(list(off), dtype=np.int64)
        self.n_cells = int(self.cell_offset[-1])
        self.levelled = False

    # -- helpers -----------------------------------------------------------
    def _stream(self):
        return ctypes.c_void_p(torch.cuda.current_stream(self.device).cuda_stream)

    def _check(self, code, ctx=0):
        if code != 0:
            c = self.ctx if ctx == 0 else ctx
            msg = self.lib.ebr_last_error(c).decode() if c else ""
            raise _lib.EBRError(code, msg)

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.ebr_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- steps ---------------------------------------------------------------
    def classify(self, tags=None):
        """Re-run the classification (no host synchronisation)."""
        t = self.tags if tags is None else tags
        self._check(self.lib.ebr_classify(self.ctx, _ptr(t), self._stream()))
        return t

    def move(self, bodies):
        """Move the bodies (same kinds and grids) and re-plan the geometry
        set; levels must be built again before the next fill."""
        if isinstance(bodies, dict):
            bodies = [bodies]
        if len(bodies) != self.B:
            raise ValueError("move needs %d bodies" % self.B)
        self._bodies = (_lib.Body * self.B)(*[_body_struct(b) for b in bodies])
        self._check(self.lib.ebr_move(self.ctx, self._bodies, _ptr(self.tags), self._stream()))
        self.levelled = False

    def build_levels(self):
        self._check(self.lib.ebr_build_levels(self.ctx, self._stream()))
        self.levelled = True

    def classify_levels(self, tags=None):
        """Re-run the classification and the levels of a levelled context in
        one call (ebr_classify_levels: for one-layer HGC the double closest
        points overlap the levels)."""
        if not self.levelled:
            raise RuntimeError("classify_levels needs a levelled context (build_levels first)")
        t = self.tags if tags is None else tags
        self._check(self.lib.ebr_classify_levels(self.ctx, _ptr(t), self._stream()))
        return t

    def counts(self):
        arr = (_lib.GeomCounts * self.B)()
        self._check(self.lib.ebr_counts(self.ctx, arr))
        return [{"n_cells": a.n_cells, "n_interface": a.n_interface, "n_ghosts": a.n_ghosts,
                 "n_levels": a.n_levels} for a in arr]

    @property
    def n_ghosts(self):
        return int(sum(c["n_ghosts"] for c in self.counts()))

    def ghost_info(self):
        ng = self.n_ghosts
        out = {
            "geom": np.zeros(ng, np.int32), "cell": np.zeros(ng, np.int64),
            "level": np.zeros(ng, np.int32), "tag": np.zeros(ng, np.int8),
            "psi": np.zeros(ng, np.float64), "normal": np.zeros((ng, 3), np.float64),
            "S": np.zeros((ng, 3), np.float64), "r": np.zeros((ng, 3), np.int32),
        }
        P = lambda a: a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
        self._check(self.lib.ebr_ghost_info(self.ctx, P(out["geom"]), P(out["cell"]), P(out["level"]),
                                            P(out["tag"]), P(out["psi"]), P(out["normal"]),
                                            P(out["S"]), P(out["r"]), self._stream()))
        return out

    def reconstruct(self, fields, bc_kinds, bc, mode="persistent"):
        F = len(fields)
        dt = fields[0].dtype
        kinds = (ctypes.c_int32 * F)(*[int(k) for k in bc_kinds])
        self._check(self.lib.ebr_reconstruct(self.ctx, F, _ptr_array(fields), kinds, _ptr_array(bc),
                                             DTYPE[dt], MODE[mode], self._stream()))
        return fields

    def forces(self, vel, p, mu, dirs, out=None):
        d = self.dim
        W = 2 * d + 2
        if out is None:
            out = torch.empty(self.B * W, dtype=torch.float64, device=self.device)
        dd = (ctypes.c_double * (2 * d))(*[float(v) for v in np.asarray(dirs, dtype=np.float64).reshape(-1)[: 2 * d]])
        self._check(self.lib.ebr_boundary_forces(self.ctx, _ptr_array(list(vel)), _ptr(p),
                                                 DTYPE[p.dtype], float(mu), dd, _ptr(out), self._stream()))
        return out.view(self.B, W)

    def adjoint(self, bc_kinds, vel_index, p_index, mu, dirs, seed, grad_fields, grad_bc,
                accumulate=False, mode="persistent"):
        F = len(bc_kinds)
        d = self.dim
        kinds = (ctypes.c_int32 * F)(*[int(k) for k in bc_kinds])
        vi = (ctypes.c_int32 * 3)(*([(-1 if v is None else int(v)) for v in vel_index] + [-1] * (3 - len(vel_index))))
        dd = (ctypes.c_double * (2 * d))(*[float(v) for v in np.asarray(dirs, dtype=np.float64).reshape(-1)[: 2 * d]])
        seed = seed.to(device=self.device, dtype=torch.float64).contiguous()
        self._check(self.lib.ebr_reconstruct_adjoint(
            self.ctx, F, kinds, vi, int(p_index), float(mu), dd, _ptr(seed),
            _ptr_array(grad_fields), _ptr_array(grad_bc), DTYPE[grad_fields[0].dtype],
            1 if accumulate else 0, MODE[mode], self._stream()))
        return grad_fields, grad_bc

    # -- many fields, field-minor layout [cells][F] ----------------------------
    def reconstruct_packed(self, fields, bc_kinds, bc):
        """Fill the ghost entries of `fields` ([cells, F], contiguous) in place;
        `bc` is [ghosts, F] in canonical ghost order."""
        F = int(fields.shape[1])
        self._packed_check(fields, F, self.n_cells)
        self._packed_check(bc, F, self.n_ghosts)
        kinds = (ctypes.c_int32 * F)(*[int(k) for k in bc_kinds])
        self._check(self.lib.ebr_reconstruct_packed(self.ctx, F, _ptr(fields), kinds, _ptr(bc),
                                                    DTYPE[fields.dtype], self._stream()))
        return fields

    def reconstruct_packed_adjoint(self, bc_kinds, cot, grad_bc):
        """Transpose of reconstruct_packed, in place on `cot` ([cells, F]):
        dJ/d(filled field) in, dJ/d(field before the fill) out; `grad_bc`
        ([ghosts, F]) receives dJ/d(boundary data)."""
        F = int(cot.shape[1])
        self._packed_check(cot, F, self.n_cells)
        self._packed_check(grad_bc, F, self.n_ghosts)
        kinds = (ctypes.c_int32 * F)(*[int(k) for k in bc_kinds])
        self._check(self.lib.ebr_reconstruct_packed_adjoint(self.ctx, F, kinds, _ptr(cot), _ptr(grad_bc),
                                                            DTYPE[cot.dtype], self._stream()))
        return cot, grad_bc

    def _packed_check(self, t, F, rows):
        if t.dim() != 2 or not t.is_contiguous() or int(t.shape[1]) != F or t.device != self.device:
            raise ValueError("packed arrays are contiguous [rows, F] tensors on %s" % self.device)
        if rows is not None and int(t.shape[0]) != rows:
            raise ValueError("packed field array needs %d rows (cells), got %d" % (rows, int(t.shape[0])))

    # -- tiled fill with a per-level exchange -----------------------------------
    def tiled_plan(self, tile):
        """Plan tiles of `tile` cells per axis (host step; before any capture)."""
        t = (ctypes.c_int32 * 3)(*([int(v) for v in tile] + [1] * (3 - len(tile))))
        self._check(self.lib.ebr_tiled_plan(self.ctx, t, self._stream()))

    def reconstruct_tiled(self, fields, bc_kinds, bc):
        F = len(fields)
        kinds = (ctypes.c_int32 * F)(*[int(k) for k in bc_kinds])
        self._check(self.lib.ebr_reconstruct_tiled(self.ctx, F, _ptr_array(fields), kinds, _ptr_array(bc),
                                                   DTYPE[fields[0].dtype], self._stream()))
        return fields

    def tiled_info(self):
        n = 8 + 256
        out = (ctypes.c_int64 * n)()
        self._check(self.lib.ebr_tiled_info(self.ctx, out, n))
        L = int(out[5])
        return {"active_tiles": int(out[0]), "tiles": int(out[1]), "sent_ghosts": int(out[2]),
                "values_exchanged": int(out[3]), "halo_values": int(out[4]), "levels": L,
                "grid_f32": int(out[6]), "grid_f64": int(out[7]),
                "sent_per_level": [int(out[8 + k]) for k in range(min(L, 256))]}

    def tiled_lists(self):
        ng = self.n_ghosts
        tile = np.zeros(ng, np.int32)
        slot = np.zeros(ng, np.int32)
        self._check(self.lib.ebr_tiled_lists(self.ctx, tile.ctypes.data_as(ctypes.c_void_p),
                                             slot.ctypes.data_as(ctypes.c_void_p)))
        return tile, slot

    def tiled_wait_test(self, spins):
        self._check(self.lib.ebr_tiled_wait_test(self.ctx, int(spins)))

    def stats(self, n_bins=60, n_levels=256):
        """Stability diagnostics (Eq. stability_alpha_max): per geometry max and
        min alpha per axis, alpha histogram over [-0.5, 1), level and r
        histograms."""
        alpha = np.zeros((self.B, 6))
        ah = np.zeros((3, n_bins), np.int64)
        lh = np.zeros(n_levels, np.int64)
        rh = np.zeros((3, 16), np.int64)
        P = lambda a: a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
        self._check(self.lib.ebr_stats(self.ctx, P(alpha), P(ah), n_bins, P(lh), n_levels, P(rh), self._stream()))
        d = self.dim
        return {"alpha_max": alpha[:, :d], "alpha_min": alpha[:, 3:3 + d], "alpha_hist": ah[:d],
                "bin_edges": np.linspace(-0.5, 1.0, n_bins + 1), "level_hist": lh, "r_hist": rh[:d]}

    def sync_status(self):
        self._check(self.lib.ebr_sync_status(self.ctx, self._stream()))

    def diagnostics(self):
        out = (ctypes.c_int64 * 12)()
        self._check(self.lib.ebr_diagnostics(self.ctx, out, 12, self._stream()))
        return {"row_fallbacks": int(out[0]), "r_max": int(out[1]), "launches": int(out[2]),
                "n_gsrc": int(out[3]),
                "packed": {"grid_levels_fill": int(out[4]), "grid_levels_adjoint": int(out[5]),
                           "tail_geometries_fill": int(out[6]), "tail_geometries_adjoint": int(out[7]),
                           "largest_tail_fill": int(out[8]), "largest_tail_adjoint": int(out[9]),
                           "fluid_targets": int(out[10])},
                "allocations": int(out[11])}

    def profile(self, enable=True):
        self._check(self.lib.ebr_profile(self.ctx, 1 if enable else 0))

    def profile_read(self, max_entries=64, keep=False):
        names = ctypes.create_string_buffer(32 * max_entries)
        ms = (ctypes.c_double * max_entries)()
        cnt = (ctypes.c_int64 * max_entries)()
        n = self.lib.ebr_profile_read(self.ctx, max_entries, names, ms, cnt, 1 if keep else 0)
        if n < 0:
            self._check(n)
        out = {}
        for k in range(min(n, max_entries)):
            nm = names.raw[32 * k: 32 * k + 32].split(b"\0", 1)[0].decode()
            out[nm] = (float(ms[k]), int(cnt[k]))
        return out

    def profile_timeline(self, max_entries=256):
        """[(name, start_ms, end_ms)] of the kept records in issue order,
        relative to the start of the first record."""
        names = ctypes.create_string_buffer(32 * max_entries)
        t0 = (ctypes.c_double * max_entries)()
        t1 = (ctypes.c_double * max_entries)()
        n = self.lib.ebr_profile_timeline(self.ctx, max_entries, names, t0, t1)
        if n < 0:
            self._check(n)
        return [(names.raw[32 * k: 32 * k + 32].split(b"\0", 1)[0].decode(), float(t0[k]), float(t1[k]))
                for k in range(min(n, max_entries))]

    # -- launch shapes ----------------------------------------------------------
    def tunable_kernels(self):
        n = int(self.lib.ebr_tunable_kernels(None, 0))
        names = ctypes.create_string_buffer(32 * n)
        self.lib.ebr_tunable_kernels(names, n)
        return [names.raw[32 * k: 32 * k + 32].split(b"\0", 1)[0].decode() for k in range(n)]

    def set_block_size(self, kernel, threads):
        self._check(self.lib.ebr_set_block_size(self.ctx, kernel.encode(), int(threads)))

    def block_size(self, kernel):
        v = int(self.lib.ebr_get_block_size(self.ctx, kernel.encode()))
        if v < 0:
            raise ValueError("no tunable kernel named %r" % kernel)
        return v

    @property
    def launches(self):
        return int(self.lib.ebr_launch_count(self.ctx))

    def drag_lift(self, fields, bcs, bc_kinds, vel_index, p_index, mu, dirs, mode="persistent"):
        """(drag, lift) per geometry [B, 2], differentiable with respect to the
        field values and the boundary data (backward = ebr_reconstruct_adjoint)."""
        return DragLift.apply(self, tuple(int(k) for k in bc_kinds), tuple(vel_index), int(p_index),
                              float(mu), tuple(np.asarray(dirs, np.float64).reshape(-1)), mode,
                              *fields, *bcs)


class DragLift(torch.autograd.Function):
    """Fill (out of place) + forces forward; the library's adjoint backward.

    The ghost entries of the input fields do not influence the result (the
    fill overwrites them), so their gradient is zero."""

    @staticmethod
    def forward(ctx, R, bc_kinds, vel_index, p_index, mu, dirs, mode, *tensors):
        F = len(bc_kinds)
        fields = [t.detach().clone() for t in tensors[:F]]
        bcs = [t.detach() for t in tensors[F:]]
        R.reconstruct(fields, bc_kinds, bcs, mode=mode)
        d = R.dim
        vel = [fields[i] if i is not None and i >= 0 else None for i in vel_index]
        out = R.forces(vel, fields[p_index], mu, np.asarray(dirs).reshape(2, d))
        ctx.R, ctx.args = R, (bc_kinds, vel_index, p_index, mu, dirs, mode)
        ctx.shapes = [(t.shape, t.dtype, t.device) for t in tensors]
        return out[:, 2 * d: 2 * d + 2].clone()

    @staticmethod
    def backward(ctx, g):
        R = ctx.R
        bc_kinds, vel_index, p_index, mu, dirs, mode = ctx.args
        F = len(bc_kinds)
        grads = [torch.zeros(s, dtype=dt, device=dv) for s, dt, dv in ctx.shapes]
        R.adjoint(bc_kinds, list(vel_index), p_index, mu, np.asarray(dirs).reshape(2, R.dim),
                  g.detach().to(torch.float64), grads[:F], grads[F:], accumulate=False, mode=mode)
        return (None,) * 7 + tuple(grads)
