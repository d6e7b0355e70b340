"""Python objects over the C ABI: a device context holding resident geometry
and batches of body pairs.  Torch tensors provide device memory and streams;
every step of the contact computation runs in ``libccm.so``."""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import abi
from .abi import check, lib, ptr


def _params(params):
    if params is None:
        return abi.default_params()
    if isinstance(params, abi.ccm_params):
        return params
    return abi.default_params(**params)


class Context:
    """``ccm_create`` / ``ccm_destroy`` plus geometry residency."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0):
        self.device = device
        h = C.c_void_p()
        check(lib().ccm_create(device, hbm_budget_bytes, C.byref(h)))
        self.handle = h

    def close(self):
        if self.handle:
            lib().ccm_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def load_geometry(self, geom) -> np.ndarray:
        """Uploads every body of a ``scenes.Geometry``; returns uint64 handles."""
        nb = geom.n_bodies
        keep = []
        descs = (abi.ccm_body_desc * nb)()
        for b in range(nb):
            p0, p1 = int(geom.body_piece_off[b]), int(geom.body_piece_off[b + 1])
            nv = np.diff(geom.piece_v_off[p0:p1 + 1]).astype(np.int32)
            nf = np.diff(geom.piece_f_off[p0:p1 + 1]).astype(np.int32)
            ne = np.diff(geom.piece_e_off[p0:p1 + 1]).astype(np.int32)
            v = np.ascontiguousarray(geom.verts[geom.piece_v_off[p0]:geom.piece_v_off[p1]], np.float32)
            f = np.ascontiguousarray(geom.planes[geom.piece_f_off[p0]:geom.piece_f_off[p1]], np.float32)
            e = np.ascontiguousarray(geom.edges[geom.piece_e_off[p0]:geom.piece_e_off[p1]], np.int32)
            keep += [nv, nf, ne, v, f, e]
            descs[b] = abi.ccm_body_desc(p1 - p0, ptr(nv), ptr(nf), ptr(ne), ptr(v), ptr(f),
                                         ptr(e) if e.size else ptr(np.zeros(2, np.int32)))
        out = np.zeros(nb, np.uint64)
        check(lib().ccm_load_geometry(self.handle, descs, nb, ptr(out)))
        return out

    def free_geometry(self, handles):
        h = np.ascontiguousarray(handles, np.uint64)
        check(lib().ccm_free_geometry(self.handle, ptr(h), len(h)))

    def output_size(self, A, B) -> int:
        A = np.ascontiguousarray(A, np.uint64)
        B = np.ascontiguousarray(B, np.uint64)
        G = C.c_int64()
        check(lib().ccm_output_size(self.handle, len(A), ptr(A), ptr(B), C.byref(G)))
        return G.value

    def batch(self, A, B) -> "Batch":
        return Batch(self, A, B)


class Batch:
    """``ccm_batch_create``: a fixed list of body pairs (A[i], B[i])."""

    def __init__(self, ctx: Context, A, B):
        self.ctx = ctx
        A = np.ascontiguousarray(A, np.uint64)
        B = np.ascontiguousarray(B, np.uint64)
        h = C.c_void_p()
        check(lib().ccm_batch_create(ctx.handle, len(A), ptr(A), ptr(B), C.byref(h)))
        self.handle = h
        n = C.c_int64()
        G = C.c_int64()
        check(lib().ccm_batch_info(h, C.byref(n), C.byref(G), None))
        self.n_pairs, self.n_groups = n.value, G.value
        self.group_offsets = np.zeros(self.n_pairs + 1, np.int64)
        check(lib().ccm_batch_info(h, None, None, ptr(self.group_offsets)))

    def get_tuning(self) -> dict:
        t = abi.ccm_tuning()
        check(lib().ccm_batch_get_tuning(self.handle, C.byref(t)))
        return {k: getattr(t, k) for k in ("item_v", "item_e", "item_vb", "item_eb", "fwd_warps")}

    def set_tuning(self, **kw):
        t = abi.ccm_tuning()
        check(lib().ccm_batch_get_tuning(self.handle, C.byref(t)))
        for k, v in kw.items():
            setattr(t, k, int(v))
        check(lib().ccm_batch_set_tuning(self.handle, C.byref(t)))

    def close(self):
        if self.handle:
            lib().ccm_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check_pose(self, p):
        import torch
        if not (p.is_cuda and p.dtype == torch.float32 and p.is_contiguous()
                and tuple(p.shape) == (self.n_pairs, 12)):
            raise ValueError(f"pose must be a contiguous cuda float32 [{self.n_pairs}, 12] tensor")

    def contacts(self, pose_a, pose_b, params=None, out=None, counters=None):
        """Group outputs y [G, 8] (d, a, p, n) as a cuda tensor."""
        import torch
        self._check_pose(pose_a)
        self._check_pose(pose_b)
        if out is None:
            out = torch.empty((self.n_groups, 8), device=pose_a.device, dtype=torch.float32)
        prm = _params(params)
        s = abi.stream_of(pose_a)
        if counters is None:
            check(lib().ccm_contacts(self.handle, ptr(pose_a), ptr(pose_b), C.byref(prm),
                                     ptr(out), s))
        else:
            check(lib().ccm_contacts_counted(self.handle, ptr(pose_a), ptr(pose_b),
                                             C.byref(prm), ptr(out), ptr(counters), s))
        return out

    def backward(self, pose_a, pose_b, ybar, direction=None, params=None, want_jvp=False,
                 out=None):
        """(grad [n,12], hvp [n,12] | None, jvp [G,8] | None) of <ybar, y> in
        the twist chart (w_A, v_A, w_B, v_B); ``out`` = preallocated
        (grad, hvp, jvp) tensors (any may be None)."""
        import torch
        self._check_pose(pose_a)
        self._check_pose(pose_b)
        dev = pose_a.device
        ybar = ybar.contiguous()
        o_g, o_h, o_j = out if out is not None else (None, None, None)
        grad = o_g if o_g is not None else torch.empty((self.n_pairs, 12), device=dev,
                                                       dtype=torch.float32)
        hvp = jvp = None
        if direction is not None:
            direction = direction.contiguous()
            hvp = o_h if o_h is not None else torch.empty((self.n_pairs, 12), device=dev,
                                                          dtype=torch.float32)
            if want_jvp:
                jvp = o_j if o_j is not None else torch.empty((self.n_groups, 8), device=dev,
                                                              dtype=torch.float32)
        prm = _params(params)
        check(lib().ccm_contacts_backward(self.handle, ptr(pose_a), ptr(pose_b), C.byref(prm),
                                          ptr(ybar), ptr(direction), ptr(grad), ptr(hvp),
                                          ptr(jvp), abi.stream_of(pose_a)))
        return grad, hvp, jvp


def scene_to_device(scene, ctx: Context, device="cuda"):
    """Loads a ``scenes.Scene`` (geometry, pairs, poses) into ``ctx``: returns
    (batch, pose_a, pose_b) with poses as cuda float32 tensors."""
    import torch
    handles = ctx.load_geometry(scene.geom)
    batch = ctx.batch(handles[scene.pair_a], handles[scene.pair_b])
    pa = torch.from_numpy(np.ascontiguousarray(scene.pose_a, np.float32)).to(device)
    pb = torch.from_numpy(np.ascontiguousarray(scene.pose_b, np.float32)).to(device)
    return batch, pa, pb
