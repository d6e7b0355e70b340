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

    def attach_splines(self, geom, handles):
        """Attaches the tricubic spline SDFs of ``geom.splines`` (a
        ``scenes.SplineSet``) to the bodies ``handles`` (``load_geometry``'s
        result for the same geometry)."""
        sp = geom.splines
        for b in range(geom.n_bodies):
            p0, p1 = int(geom.body_piece_off[b]), int(geom.body_piece_off[b + 1])
            dims = np.ascontiguousarray(sp.dims[p0:p1, :3], np.int32)
            grid = np.ascontiguousarray(sp.grid[p0:p1], np.float32)
            r0 = int(sp.dims[p0, 3])
            r1 = int(sp.dims[p1, 3]) if p1 < len(sp.dims) else len(sp.coef)
            coef = np.ascontiguousarray(sp.coef[r0:r1], np.float32)
            desc = abi.ccm_spline_desc(ptr(grid), ptr(dims), ptr(coef))
            check(lib().ccm_attach_splines(self.handle, C.c_uint64(int(handles[b])),
                                           C.byref(desc)))

    def build_voxel_grids(self, voxels: int = 8):
        """``ccm_build_voxel_grids``: broad-phase voxel grids of every loaded
        piece (used by the forward with the CCM_FLAG_VOXEL_CULL flag)."""
        check(lib().ccm_build_voxel_grids(self.handle, int(voxels)))

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
        return {k: getattr(t, k) for k in ("item_v", "item_e", "item_vb", "item_eb", "fwd_warps",
                                           "groups", "stage_planes", "stage_verts", "groups_b",
                                           "flat_records", "stage_tma", "stage_wait",
                                           "flat_forward", "pdl")}

    def set_tuning(self, **kw):
        t = abi.ccm_tuning()
        check(lib().ccm_batch_get_tuning(self.handle, C.byref(t)))
        for k, v in kw.items():
            setattr(t, k, int(v))
        check(lib().ccm_batch_set_tuning(self.handle, C.byref(t)))

    def check(self, stream=None):
        """``ccm_batch_check``: waits for the stream and raises CcmError
        (CCM_ERR_TIMEOUT) if a kernel of the batch stopped on a bounded wait."""
        import torch
        s = stream if stream is not None else torch.cuda.current_stream()
        check(lib().ccm_batch_check(self.handle, C.c_void_p(s.cuda_stream)))

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

    def saved_buffer(self, device="cuda"):
        """An uninitialised [G, CCM_SAVED_FLOATS] record for ``contacts(saved=...)``."""
        import torch
        return torch.empty((self.n_groups, abi.CCM_SAVED_FLOATS), device=device,
                           dtype=torch.float32)

    def contacts(self, pose_a, pose_b, params=None, out=None, counters=None, saved=None):
        """Group outputs y [G, 8] (d, a, p, n) as a cuda tensor.  ``saved``: a
        ``saved_buffer()`` that receives the record ``backward(saved=...)``
        uses (``ccm_contacts_save``)."""
        import torch
        self._check_pose(pose_a)
        self._check_pose(pose_b)
        if out is None:
            out = torch.empty((self.n_groups, 8), device=pose_a.device, dtype=torch.float32)
        prm = _params(params)
        s = abi.stream_of(pose_a)
        if counters is not None:
            check(lib().ccm_contacts_counted(self.handle, ptr(pose_a), ptr(pose_b),
                                             C.byref(prm), ptr(out), ptr(counters), s))
        elif saved is not None:
            self._check_saved(saved)
            check(lib().ccm_contacts_save(self.handle, ptr(pose_a), ptr(pose_b), C.byref(prm),
                                          ptr(out), ptr(saved), s))
        else:
            check(lib().ccm_contacts(self.handle, ptr(pose_a), ptr(pose_b), C.byref(prm),
                                     ptr(out), s))
        return out

    def _check_saved(self, saved):
        import torch
        if not (saved.is_cuda and saved.dtype == torch.float32 and saved.is_contiguous()
                and tuple(saved.shape) == (self.n_groups, abi.CCM_SAVED_FLOATS)):
            raise ValueError("saved must be a contiguous cuda float32 "
                             f"[{self.n_groups}, {abi.CCM_SAVED_FLOATS}] tensor")

    def backward(self, pose_a, pose_b, ybar, direction=None, params=None, want_jvp=False,
                 out=None, saved=None, counters=None):
        """(grad [n,12], hvp [n,12] | None, jvp [G,8] | None) of <ybar, y> in
        the twist chart (w_A, v_A, w_B, v_B); ``out`` = preallocated
        (grad, hvp, jvp) tensors (any may be None); ``saved`` = the record of
        a ``contacts(saved=...)`` call with the same poses and params."""
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
        if saved is not None:
            self._check_saved(saved)
        if counters is not None:
            check(lib().ccm_contacts_backward_counted(self.handle, ptr(pose_a), ptr(pose_b),
                                                      C.byref(prm), ptr(saved), ptr(ybar),
                                                      ptr(direction), ptr(grad), ptr(hvp),
                                                      ptr(jvp), ptr(counters),
                                                      abi.stream_of(pose_a)))
        elif saved is None:
            check(lib().ccm_contacts_backward(self.handle, ptr(pose_a), ptr(pose_b),
                                              C.byref(prm), ptr(ybar), ptr(direction),
                                              ptr(grad), ptr(hvp), ptr(jvp),
                                              abi.stream_of(pose_a)))
        else:
            check(lib().ccm_contacts_backward_saved(self.handle, ptr(pose_a), ptr(pose_b),
                                                    C.byref(prm), ptr(saved), ptr(ybar),
                                                    ptr(direction), ptr(grad), ptr(hvp),
                                                    ptr(jvp), abi.stream_of(pose_a)))
        return grad, hvp, jvp

    def step_host(self, pose_a, pose_b, ybar=None, direction=None, params=None,
                  want_jvp=False, out=None, stream=None):
        """One step from host tensors (``ccm_contacts_step_host``): forward
        (y), then with ``ybar`` the gradient and with ``direction`` H u and
        (``want_jvp``) J u, with the host<->device copies overlapped with the
        kernels.  Inputs are contiguous CPU float32 tensors (pinned for
        asynchronous copies); returns CPU tensors (y, grad, hvp, jvp), None
        where not asked, written once ``stream`` (default: the current cuda
        stream) reaches this point -- synchronize before reading them.
        ``out``: preallocated (y, grad, hvp, jvp) CPU tensors (any may be None)."""
        import torch

        def host(t, shape, name):
            if t is None:
                return None
            if not (t.device.type == "cpu" and t.dtype == torch.float32 and t.is_contiguous()
                    and tuple(t.shape) == shape):
                raise ValueError(f"{name} must be a contiguous CPU float32 {list(shape)} tensor")
            return t

        P, G8 = (self.n_pairs, 12), (self.n_groups, 8)
        pose_a, pose_b = host(pose_a, P, "pose_a"), host(pose_b, P, "pose_b")
        ybar, direction = host(ybar, G8, "ybar"), host(direction, P, "direction")
        o = list(out) if out is not None else [None] * 4

        def new(i, shape):
            return o[i] if o[i] is not None else torch.empty(shape, pin_memory=True)
        y = host(new(0, G8), G8, "y")
        grad = host(new(1, P), P, "grad") if ybar is not None else None
        hvp = host(new(2, P), P, "hvp") if direction is not None else None
        jvp = host(new(3, G8), G8, "jvp") if direction is not None and want_jvp else None
        prm = _params(params)
        s = stream if stream is not None else torch.cuda.current_stream()
        check(lib().ccm_contacts_step_host(self.handle, ptr(pose_a), ptr(pose_b), C.byref(prm),
                                           ptr(ybar), ptr(direction), ptr(y), ptr(grad),
                                           ptr(hvp), ptr(jvp), C.c_void_p(s.cuda_stream)))
        return y, grad, hvp, jvp


def scene_to_device(scene, ctx: Context, device="cuda"):
    """Loads a ``scenes.Scene`` (geometry, pairs, poses) into ``ctx``: returns
    (batch, pose_a, pose_b) with poses as cuda float32 tensors."""
    import torch
    handles = ctx.load_geometry(scene.geom)
    batch = ctx.batch(handles[scene.pair_a], handles[scene.pair_b])
    pa = torch.from_numpy(np.ascontiguousarray(scene.pose_a, np.float32)).to(device)
    pb = torch.from_numpy(np.ascontiguousarray(scene.pose_b, np.float32)).to(device)
    return batch, pa, pb


class Server:
    """Continuous batching over a context (``ccm_serve_start`` .. ``ccm_serve_stop``).

    ``submit`` queues the contacts (and optionally the pose gradient) of a list
    of body pairs and returns a ticket; ``poll`` reports completion without
    blocking.  The tensors of a request are kept alive here until its ticket is
    retired."""

    def __init__(self, ctx: Context, params=None, tuning: dict | None = None, **capacities):
        self.ctx = ctx
        cfg = abi.default_serve_config(**capacities)
        cfg.params = _params(params)
        for k, v in (tuning or {}).items():
            setattr(cfg.tuning, k, int(v))
        check(lib().ccm_serve_start(ctx.handle, C.byref(cfg)))
        self.config = cfg
        self._live = {}

    def submit(self, A, B, pose_a, pose_b, ybar=None, y=None, grad=None, sync=True):
        """Queues one request.  pose_a / pose_b: cuda float32 [n, 12]; ybar:
        cuda float32 [G, 8] for the gradient, else None.  ``sync`` waits for
        the current stream first so that the poses hold their values.
        Returns (ticket, y, grad); y and grad are filled once ``poll`` says done."""
        import torch
        A = np.ascontiguousarray(A, np.uint64)
        B = np.ascontiguousarray(B, np.uint64)
        n = len(A)
        dev = pose_a.device
        for p in (pose_a, pose_b):
            if not (p.is_cuda and p.dtype == torch.float32 and p.is_contiguous()
                    and tuple(p.shape) == (n, 12)):
                raise ValueError(f"pose must be a contiguous cuda float32 [{n}, 12] tensor")
        if y is None:
            y = torch.empty((self.ctx.output_size(A, B), 8), device=dev, dtype=torch.float32)
        if ybar is not None:
            ybar = ybar.contiguous()
            if grad is None:
                grad = torch.empty((n, 12), device=dev, dtype=torch.float32)
        if sync:
            torch.cuda.current_stream(dev).synchronize()
        req = abi.ccm_request(n, ptr(A), ptr(B), ptr(pose_a), ptr(pose_b), ptr(y), ptr(ybar),
                              ptr(grad) if ybar is not None else None)
        t = C.c_uint64()
        check(lib().ccm_submit(self.ctx.handle, C.byref(req), C.byref(t)))
        self._live[t.value] = (pose_a, pose_b, y, ybar, grad)
        return t.value, y, grad

    def poll(self, ticket):
        """(done, latency in seconds or None)."""
        done = C.c_int()
        lat = C.c_double()
        check(lib().ccm_poll(self.ctx.handle, C.c_uint64(ticket), C.byref(done), C.byref(lat)))
        if done.value:
            self._live.pop(ticket, None)
            return True, lat.value
        return False, None

    def completed(self, max_n=4096):
        """Retires the requests completed so far, in completion order:
        a list of (ticket, latency in seconds)."""
        t = np.zeros(max_n, np.uint64)
        lat = np.zeros(max_n, np.float64)
        n = C.c_int64()
        check(lib().ccm_poll_completed(self.ctx.handle, ptr(t), ptr(lat), max_n, C.byref(n)))
        out = list(zip(t[:n.value].tolist(), lat[:n.value].tolist()))
        for tk, _ in out:
            self._live.pop(tk, None)
        return out

    def wait(self, ticket, timeout_s=60.0):
        """Polls until done; returns the latency.  Raises TimeoutError."""
        import time
        t_end = time.perf_counter() + timeout_s
        while True:
            done, lat = self.poll(ticket)
            if done:
                return lat
            if time.perf_counter() > t_end:
                raise TimeoutError(f"ticket {ticket} not done after {timeout_s} s")
            time.sleep(20e-6)

    def stats(self):
        c = abi.ccm_serve_counters()
        check(lib().ccm_serve_stats(self.ctx.handle, C.byref(c)))
        return {k: getattr(c, k) for k, _ in abi.ccm_serve_counters._fields_}

    def hold(self, on: bool):
        """While held, queued requests form no new wave."""
        check(lib().ccm_serve_hold(self.ctx.handle, 1 if on else 0))

    def close(self):
        if self.ctx is not None and self.ctx.handle:
            check(lib().ccm_serve_stop(self.ctx.handle))
        self._live.clear()
        self.ctx = None
