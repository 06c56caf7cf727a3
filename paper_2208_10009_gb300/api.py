"""Python front end of the SBR library: thin wrappers over the C ABI (``include/sbr.h``).

Every step of the hot path runs in the CUDA library; this module only marshals
arguments.  Device memory comes from PyTorch's caching allocator through the ABI's
allocator callbacks, and work is enqueued on a PyTorch CUDA stream.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np
import torch

from . import _binding as B


class SbrError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{B.STATUS.get(status, status)}: {msg}")
        self.status = status


def _ptr(t) -> int | None:
    if t is None:
        return None
    if isinstance(t, torch.Tensor):
        return t.data_ptr()
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    raise TypeError(type(t))


def _host_f32(a, cols=3):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float32).reshape(-1, cols))
    return a


@dataclass
class LaunchConfig:
    n_div: int
    max_order: int
    rx_angle_scale: float = 1.0
    grid_blocks: int = 0
    block_threads: int = 0


class Scene:
    def __init__(self, ctx: "Context", handle: int, nf: int):
        self.ctx, self.handle, self.nf = ctx, handle, nf

    def info(self) -> dict:
        inf = B.SceneInfo()
        self.ctx._check(self.ctx.lib.sbr_scene_get_info(self.handle, ctypes.byref(inf)))
        return {f: (list(getattr(inf, f)) if f.startswith("bbox") else getattr(inf, f)) for f, _ in inf._fields_}

    def wedges(self):
        """The scene's wedges (order-1 diffraction): ends (W, 2, 3) float32 and face
        pairs (W, 2) int32, in wedge-id order."""
        cnt = ctypes.c_int64(0)
        self.ctx._check(self.ctx.lib.sbr_scene_wedges(self.handle, None, None, 0, ctypes.byref(cnt)))
        n = cnt.value
        ab = np.zeros((max(n, 1), 6), np.float32)
        fc = np.zeros((max(n, 1), 2), np.int32)
        self.ctx._check(self.ctx.lib.sbr_scene_wedges(self.handle, ab.ctypes.data, fc.ctypes.data, n,
                                                      ctypes.byref(cnt)))
        return ab[:n].reshape(-1, 2, 3), fc[:n]

    def close(self):
        if self.handle:
            self.ctx.lib.sbr_scene_destroy(self.ctx.handle, self.handle)
            self.handle = None


class RxSet:
    def __init__(self, ctx: "Context", handle: int, n: int):
        self.ctx, self.handle, self.n = ctx, handle, n

    def close(self):
        if self.handle:
            self.ctx.lib.sbr_rx_destroy(self.ctx.handle, self.handle)
            self.handle = None


class Paths:
    def __init__(self, ctx: "Context", handle: int, record_cap: int, path_cap: int):
        self.ctx, self.handle = ctx, handle
        self.record_cap, self.path_cap = record_cap, path_cap

    def close(self):
        if self.handle:
            self.ctx.lib.sbr_paths_destroy(self.ctx.handle, self.handle)
            self.handle = None


class Context:
    """One library context on one CUDA device and stream."""

    def __init__(self, device: int = 0, stream: torch.cuda.Stream | None = None, torch_allocator: bool = True,
                 checked: bool = False):
        """`checked` runs the bounds-checked build of the library (SBR_CHECKED)."""
        if not torch.cuda.is_available():
            raise SbrError(3, "no CUDA device: the SBR library has no CPU path")
        self.lib = B.load(checked=checked)
        self.device = device
        self.stream = stream or torch.cuda.current_stream(device)
        self._keep = []
        if torch_allocator:
            dev = device

            def _alloc(nbytes, stream, user):
                try:
                    return torch.cuda.caching_allocator_alloc(int(nbytes), dev, int(stream or 0))
                except Exception:
                    return None

            def _free(ptr, nbytes, stream, user):
                try:
                    torch.cuda.caching_allocator_delete(int(ptr))
                except Exception:
                    pass

            a, f = B.ALLOC_FN(_alloc), B.FREE_FN(_free)
            self._keep += [a, f]
        else:
            a, f = B.ALLOC_FN(), B.FREE_FN()
        h = ctypes.c_void_p()
        with torch.cuda.device(device):
            st = self.lib.sbr_ctx_create(device, ctypes.c_void_p(self.stream.cuda_stream), a, f, None, ctypes.byref(h))
        if st != 0:
            raise SbrError(st, "sbr_ctx_create failed")
        self.handle = h.value
        self.num_sms = self.lib.sbr_ctx_num_sms(self.handle)

    # ------------------------------------------------------------------ helpers
    def _check(self, st: int):
        if st != 0:
            msg = self.lib.sbr_last_error(self.handle) if getattr(self, "handle", None) else b""
            raise SbrError(st, (msg or b"").decode())

    def set_stream(self, stream: torch.cuda.Stream):
        self.stream = stream
        self._check(self.lib.sbr_ctx_set_stream(self.handle, ctypes.c_void_p(stream.cuda_stream)))

    def close(self):
        if getattr(self, "handle", None):
            self.lib.sbr_ctx_destroy(self.handle)
            self.handle = None

    # ------------------------------------------------------------------ geometry
    def raygen(self, n_div: int, out: torch.Tensor | None = None) -> torch.Tensor:
        N = self.lib.sbr_num_rays(n_div)
        if out is None:
            out = torch.empty((N, 4), dtype=torch.float32, device=f"cuda:{self.device}")
        self._check(self.lib.sbr_raygen(self.handle, n_div, _ptr(out), out.shape[0]))
        return out

    def raygen_equidistant(self, n_div: int, poly: int = 20, out: torch.Tensor | None = None) -> torch.Tensor:
        """§II.A equidistant division on the icosahedron (20) or octahedron (8)."""
        N = self.lib.sbr_num_rays_launcher(n_div, poly)
        if out is None:
            out = torch.empty((max(N, 1), 4), dtype=torch.float32, device=f"cuda:{self.device}")
        self._check(self.lib.sbr_raygen_equidistant(self.handle, n_div, poly, _ptr(out), out.shape[0]))
        return out

    def scene_upload(self, verts, tris, tri_face, face_eps=None, nf=None) -> Scene:
        v = _host_f32(verts)
        t = np.ascontiguousarray(np.asarray(tris, np.int32).reshape(-1, 3))
        f = np.ascontiguousarray(np.asarray(tri_face, np.int32).reshape(-1))
        nf = int(nf if nf is not None else (f.max() + 1 if len(f) else 0))
        e = None if face_eps is None else np.ascontiguousarray(np.asarray(face_eps, np.float32))
        h = ctypes.c_void_p()
        self._check(self.lib.sbr_scene_upload(
            self.handle, v.ctypes.data_as(B._pf), len(v), t.ctypes.data_as(B._pi32), f.ctypes.data_as(B._pi32),
            len(t), None if e is None else e.ctypes.data_as(B._pf), nf, ctypes.byref(h)))
        return Scene(self, h.value, nf)

    def scene_from(self, sc) -> Scene:
        return self.scene_upload(sc.verts, sc.tris, sc.tri_face, sc.face_eps, sc.nf)

    def rx_upload(self, rx) -> RxSet:
        if isinstance(rx, torch.Tensor):
            r = rx.contiguous().float()
            n = r.numel() // 3
            p = r.data_ptr()
        else:
            r = _host_f32(rx)
            n = len(r)
            p = r.ctypes.data
        h = ctypes.c_void_p()
        self._check(self.lib.sbr_rx_upload(self.handle, p, n, ctypes.byref(h)))
        return RxSet(self, h.value, n)

    def paths_create(self, record_cap: int, path_cap: int) -> Paths:
        h = ctypes.c_void_p()
        self._check(self.lib.sbr_paths_create(self.handle, record_cap, path_cap, ctypes.byref(h)))
        return Paths(self, h.value, record_cap, path_cap)

    # ------------------------------------------------------------------ hot path
    def launch(self, scene: Scene, tx, rx: RxSet, paths: Paths, n_div: int, max_order: int,
               rx_angle_scale: float = 1.0, sync: bool = False, dump_stride: int = 0,
               dump: torch.Tensor | None = None, grid_blocks: int = 0, block_threads: int = 0,
               timing: bool = False, refill_min: int = 0, launcher: int = 0, diffraction: bool = False,
               ray_range: tuple[int, int] | None = None, records_only: bool = False, id_order: bool = False):
        """a1-a5: ray generation, trace with reception, double-count removal.  `tx` is an
        (ntx, 3) array on the host (numpy) or the device (torch).  `diffraction` adds the
        order-1 diffraction search.  `ray_range` = (begin, end) traces only those ray ids of
        every Tx; `records_only` stops before double-count removal (read the records with
        `records`).  `id_order` makes the trace take the rays in lattice id order instead of
        the default compact tiles of directions (the same results)."""
        if isinstance(tx, torch.Tensor):
            txp, ntx = tx.data_ptr(), tx.numel() // 3
            keep = tx
        else:
            keep = _host_f32(tx)
            txp, ntx = keep.ctypes.data, len(keep)
        flags = ((B.LAUNCH_SYNC if sync else 0) | (B.LAUNCH_TIMING if timing else 0) |
                 (B.LAUNCH_DIFFRACTION if diffraction else 0) | (B.LAUNCH_RAY_RANGE if ray_range else 0) |
                 (B.LAUNCH_RECORDS_ONLY if records_only else 0) | (B.LAUNCH_ID_ORDER if id_order else 0))
        rb, re_ = (int(ray_range[0]), int(ray_range[1])) if ray_range else (0, 0)
        prm = B.LaunchParams(n_div, max_order, rx_angle_scale, flags, dump_stride,
                             _ptr(dump), 0 if dump is None else dump.numel(), grid_blocks, block_threads,
                             refill_min, launcher, rb, re_)
        self._check(self.lib.sbr_launch(self.handle, scene.handle, txp, ntx, rx.handle, ctypes.byref(prm),
                                        paths.handle))
        del keep

    def launch_stats(self, paths: Paths) -> dict:
        s = B.LaunchStats()
        self._check(self.lib.sbr_launch_get_stats(self.handle, paths.handle, ctypes.byref(s)))
        return {f: getattr(s, f) for f, _ in s._fields_}

    @staticmethod
    def _refine_params(max_iters, subrays, target, fp64_below, freq, ptx_dbm, choice_log):
        return B.RefineParams(max_iters, subrays, target, fp64_below, freq, ptx_dbm, _ptr(choice_log))

    def refine(self, scene: Scene, paths: Paths, max_iters: int, subrays: int = 9, target: float = 0.0,
               fp64_below: float = 1e-5, freq: float = 2.4e9, ptx_dbm: float = 0.0, choice_log=None):
        """a6-a8, plain form: one thread per path."""
        prm = self._refine_params(max_iters, subrays, target, fp64_below, freq, ptx_dbm, choice_log)
        self._check(self.lib.sbr_refine(self.handle, scene.handle, paths.handle, ctypes.byref(prm)))

    def refine_pair(self, scene: Scene, paths: Paths, tx: int, rx: int, max_iters: int, subrays: int = 9,
                    target: float = 0.0, fp64_below: float = 1e-5, freq: float = 2.4e9, ptx_dbm: float = 0.0):
        prm = self._refine_params(max_iters, subrays, target, fp64_below, freq, ptx_dbm, None)
        self._check(self.lib.sbr_refine_pair(self.handle, scene.handle, paths.handle, tx, rx, ctypes.byref(prm)))

    def batch_refine(self, scene: Scene, paths: Paths, max_iters: int, subrays: int = 9, target: float = 0.0,
                     fp64_below: float = 1e-5, freq: float = 2.4e9, ptx_dbm: float = 0.0, choice_log=None,
                     block_threads: int = 0, blocks_per_sm: int = 0, lanes_per_path: int = 0):
        """a9: persistent work-queue refinement of all pairs' paths in one launch."""
        prm = self._refine_params(max_iters, subrays, target, fp64_below, freq, ptx_dbm, choice_log)
        cfg = B.BatchConfig(block_threads, blocks_per_sm, lanes_per_path)
        self._check(self.lib.sbr_batch_refine(self.handle, scene.handle, paths.handle, ctypes.byref(prm),
                                              ctypes.byref(cfg)))

    def paths_nonfinite(self, paths: Paths) -> int:
        """Valid paths with a non-finite output (device scan; 0 when the outputs are sound)."""
        n = ctypes.c_int64()
        self._check(self.lib.sbr_paths_nonfinite(self.handle, paths.handle, ctypes.byref(n)))
        return n.value

    def paths_count(self, paths: Paths) -> int:
        n = ctypes.c_int64()
        self._check(self.lib.sbr_paths_count(self.handle, paths.handle, ctypes.byref(n)))
        return n.value

    def query(self, paths: Paths, out: np.ndarray | torch.Tensor | None = None):
        """Copy the path records to the host (numpy structured array, PATH_DTYPE) or into a
        given buffer (pinned host numpy / device torch uint8 of 128 bytes per record)."""
        if out is None:
            n = self.paths_count(paths)
            out = np.zeros(n, B.PATH_DTYPE)
            cap = n
        elif isinstance(out, torch.Tensor):
            cap = out.numel() // 128
        else:
            cap = len(out)
        w = ctypes.c_int64()
        self._check(self.lib.sbr_query(self.handle, paths.handle, _ptr(out) if cap else None, cap, ctypes.byref(w)))
        return out[: w.value] if not isinstance(out, torch.Tensor) else (out, w.value)

    def records(self, paths: Paths, out: torch.Tensor | None = None):
        """The reception records of the container's last launch (before double-count
        removal): a numpy RECORD_DTYPE array, or (out, count) when `out` is a device uint8
        tensor of 64 bytes per record."""
        if out is None:
            n = int(self.launch_stats(paths)["records"])
            out = np.zeros(min(n, paths.record_cap), B.RECORD_DTYPE)
            cap = len(out)
        else:
            cap = out.numel() // 64
        w = ctypes.c_int64()
        self._check(self.lib.sbr_records_read(self.handle, paths.handle, _ptr(out) if cap else None, cap,
                                              ctypes.byref(w)))
        return out[: w.value] if not isinstance(out, torch.Tensor) else (out, w.value)

    def records_dedup(self, paths: Paths, records, count: int | None = None, rank: int = 0, world: int = 1):
        """a5 on a given record set (host RECORD_DTYPE array or device uint8 tensor of 64-byte
        records): the container's paths become the unique paths of the (tx, rx) pairs that
        shard `rank` of `world` owns ((tx * nrx + rx) % world == rank)."""
        if isinstance(records, torch.Tensor):
            n = records.numel() // 64 if count is None else count
            p = records.data_ptr()
        else:
            records = np.ascontiguousarray(records.astype(B.RECORD_DTYPE, copy=False))
            n = len(records) if count is None else count
            p = records.ctypes.data
        self._check(self.lib.sbr_records_dedup(self.handle, paths.handle, p if n else None, n, rank, world))

    def paths_import(self, paths: Paths, records: np.ndarray, tx, rx: RxSet, n_div: int):
        recs = np.ascontiguousarray(records.astype(B.PATH_DTYPE, copy=False))
        t = _host_f32(tx)
        self._check(self.lib.sbr_paths_import(self.handle, paths.handle, recs.ctypes.data if len(recs) else None,
                                              len(recs), t.ctypes.data, len(t), rx.handle, n_div))

    # ------------------------------------------------------------------ a10
    def unfold_fwd(self, scene: Scene, tx, rx, az_el, faces, order, out=None):
        n = tx.shape[0]
        if out is None:
            out = torch.empty((n, 8), dtype=torch.float32, device=tx.device)
        self._check(self.lib.sbr_unfold_fwd(self.handle, scene.handle, n, _ptr(tx), _ptr(rx), _ptr(az_el), _ptr(faces),
                                            _ptr(order), _ptr(out)))
        return out

    def unfold_bwd(self, scene: Scene, tx, rx, az_el, faces, order, grad_out):
        n = tx.shape[0]
        g_tx = torch.empty_like(tx)
        g_rx = torch.empty_like(rx)
        g_ae = torch.empty_like(az_el)
        self._check(self.lib.sbr_unfold_bwd(self.handle, scene.handle, n, _ptr(tx), _ptr(rx), _ptr(az_el),
                                            _ptr(faces), _ptr(order), _ptr(grad_out), _ptr(g_tx), _ptr(g_rx),
                                            _ptr(g_ae)))
        return g_tx, g_rx, g_ae


# ---------------------------------------------------------------------------- host helpers
def num_rays(n_div: int) -> int:
    return B.load().sbr_num_rays(n_div)


def theta_launch(n_div: int) -> float:
    return B.load().sbr_theta_launch(n_div)


def subray_pattern(K: int):
    rho = (ctypes.c_double * 16)()
    phi = (ctypes.c_double * 16)()
    s = ctypes.c_double()
    st = B.load().sbr_subray_pattern(K, rho, phi, ctypes.byref(s))
    if st != 0:
        raise SbrError(st, f"no sub-ray pattern for K={K}")
    return np.array(rho[:K]), np.array(phi[:K]), s.value
