"""Python binding of libdpv.so (include/dpv.h): argument marshalling only.

Every step of the render and its adjoint runs in the CUDA library; this module
converts Python/torch arguments to the C ABI and wraps device pointers the
library returns as zero-copy torch tensors.  PyTorch provides device memory
and streams.  If libdpv.so is missing the import of the library raises: there
is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Iterable, List, Optional, Sequence

import numpy as np
import torch

from . import build as _build

DTYPES = {"f32": 0, "f16": 1, "bf16": 2, "fp8": 3}
TORCH_STORAGE = {0: torch.float32, 1: torch.float16, 2: torch.bfloat16, 3: torch.float8_e4m3fn}
KEY_EMPTY = 2 ** 31 - 1
FRAME_ORDER = 1
FRAME_STAGED = 2
FRAME_LINEAR = 4
FRAME_PERSISTENT = 8
FRAME_GRAPH = 16
FRAME_CELL = 32
FRAME_QUAD = 64
FRAME_ISO = 128
FRAME_ORDERED = 256
FRAME_SKIP = 512
FRAME_DEEP = 1024
DEEP_MAX = 4
FRAME_SHADOW = 2048
GATHER_FLAGS = {"auto": 0, "cell": FRAME_CELL, "quad": FRAME_QUAD, "linear": FRAME_LINEAR}


def gather_of(flags: int) -> str:
    """Gather layout name of frame flags (as dpvAutotune returns them)."""
    if flags & FRAME_LINEAR:
        return "linear"
    if flags & FRAME_CELL:
        return "cell"
    if flags & FRAME_QUAD:
        return "quad"
    return "auto"
STATUS = {0: "DPV_OK", 1: "DPV_ERR_INVALID_ARG", 2: "DPV_ERR_STATE", 3: "DPV_ERR_OUT_OF_MEMORY",
          4: "DPV_ERR_CUDA", 5: "DPV_ERR_TIMEOUT", 6: "DPV_ERR_UNSUPPORTED"}

EXPORTS = ["dpvCreateDevice", "dpvSetVolumeGeometry", "dpvCommitBrick", "dpvSetTransferFunction", "dpvSetCameras",
           "dpvSetFrame", "dpvRenderFrame", "dpvFrameReady", "dpvMapFrame", "dpvUnmapFrame", "dpvCopyFrame",
           "dpvMapFragments", "dpvUnmapFragments", "dpvReadFragments", "dpvReadDeepFragments", "dpvReadBrick", "dpvMapOrder", "dpvBackward", "dpvGetStats", "dpvResetStats", "dpvSetProfiling", "dpvGetLastError",
           "dpvRelease", "dpvRenderNoAlloc", "dpvAutotune", "dpvSetLight", "dpvCopyFrameAsync", "dpvCopyWait"]


class DPVError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))
        self.status = status


class BrickDesc(C.Structure):
    _fields_ = [("owned_lo", C.c_int * 3), ("owned_hi", C.c_int * 3), ("storage", C.c_int), ("scale", C.c_float),
                ("src_dtype", C.c_int), ("data", C.c_void_p), ("data_lo", C.c_int * 3), ("data_dims", C.c_int * 3),
                ("data_on_device", C.c_int)]


class CameraDesc(C.Structure):
    _fields_ = [("eye", C.c_float * 3), ("center", C.c_float * 3), ("up", C.c_float * 3), ("fovy_deg", C.c_float)]


class FrameDesc(C.Structure):
    _fields_ = [("width", C.c_int), ("height", C.c_int), ("step_voxels", C.c_float), ("sigma_max", C.c_float),
                ("ert_threshold", C.c_float), ("tile_w", C.c_int), ("tile_h", C.c_int), ("flags", C.c_int),
                ("iso_value", C.c_float)]


class TuneResult(C.Structure):
    _fields_ = [("tile_w", C.c_int), ("tile_h", C.c_int), ("flags", C.c_int), ("ms", C.c_float),
                ("candidates", C.c_int)]


class NoAllocBrick(C.Structure):
    _fields_ = [("owned_lo", C.c_int * 3), ("owned_hi", C.c_int * 3), ("data", C.c_void_p), ("scale", C.c_float)]


class NoAllocScene(C.Structure):
    _fields_ = [("dims", C.c_int * 3), ("origin", C.c_float * 3), ("spacing", C.c_float), ("num_ranks", C.c_int),
                ("bricks", C.POINTER(NoAllocBrick)), ("storage", C.c_int), ("tf_rgba", C.c_void_p), ("tf_n", C.c_int),
                ("vmin", C.c_float), ("vmax", C.c_float)]


STAGES = ["cull", "march", "composite", "composite_bwd", "march_bwd", "face"]


class Stats(C.Structure):
    _fields_ = [("samples_forward", C.c_uint64), ("samples_backward", C.c_uint64), ("work_items", C.c_uint64),
                ("fragment_bytes", C.c_uint64), ("error_flags", C.c_uint32), ("max_fragments", C.c_uint32),
                ("stage_ms", C.c_double * 6), ("stage_calls", C.c_uint32 * 6), ("kernel_launches", C.c_uint64),
                ("graph_launches", C.c_uint64), ("samples_shadow", C.c_uint64)]


_lib = None


def library_path() -> str:
    return _build.LIB


def load(path: Optional[str] = None):
    """Load libdpv.so (built by build.build()); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or _build.LIB
    if not os.path.exists(p):
        raise RuntimeError("libdpv.so is not built (%s): run paper_2407_00179_b300.build.build()" % p)
    lib = C.CDLL(p)
    V = C.c_void_p
    I = C.c_int
    sig = {
        "dpvCreateDevice": [I, I, V, C.POINTER(V)],
        "dpvSetVolumeGeometry": [V, C.POINTER(C.c_int), C.POINTER(C.c_float), C.c_float],
        "dpvCommitBrick": [V, I, C.POINTER(BrickDesc)],
        "dpvSetTransferFunction": [V, V, I, C.c_float, C.c_float, I],
        "dpvSetCameras": [V, C.POINTER(CameraDesc), I],
        "dpvSetLight": [V, C.POINTER(C.c_float), C.c_float, C.c_float],
        "dpvSetFrame": [V, C.POINTER(FrameDesc)],
        "dpvRenderFrame": [V],
        "dpvFrameReady": [V, I, C.POINTER(C.c_int)],
        "dpvMapFrame": [V, I, C.POINTER(V), C.POINTER(V)],
        "dpvUnmapFrame": [V, I],
        "dpvCopyFrame": [V, I, V, V],
        "dpvCopyFrameAsync": [V, I, V, V],
        "dpvCopyWait": [V],
        "dpvMapFragments": [V, I, I, C.POINTER(V)],
        "dpvUnmapFragments": [V, I, I],
        "dpvReadFragments": [V, I, I, V, V],
        "dpvReadDeepFragments": [V, I, I, I, V, V],
        "dpvMapOrder": [V, I, C.POINTER(V), C.POINTER(C.c_int)],
        "dpvReadBrick": [V, I, V, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_float)],
        "dpvBackward": [V, V, V, V],
        "dpvGetStats": [V, C.POINTER(Stats)],
        "dpvResetStats": [V],
        "dpvSetProfiling": [V, I],
        "dpvAutotune": [V, I, C.POINTER(TuneResult)],
        "dpvRenderNoAlloc": [C.POINTER(NoAllocScene), C.POINTER(CameraDesc), C.POINTER(FrameDesc), V, V, V],
        "dpvRelease": [V],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = C.c_int
    lib.dpvGetLastError.argtypes = []
    lib.dpvGetLastError.restype = C.c_char_p
    _lib = lib
    return lib


def _check(status: int):
    if status != 0:
        raise DPVError(status, load().dpvGetLastError().decode())


class _CudaArray:
    """Minimal __cuda_array_interface__ holder for a device pointer."""

    def __init__(self, ptr: int, shape, typestr: str):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr, "data": (int(ptr), False),
                                         "version": 3, "strides": None, "stream": None}


def _wrap(ptr: int, shape, dtype: torch.dtype, device) -> torch.Tensor:
    ts = {torch.float32: "<f4", torch.int32: "<i4", torch.uint8: "|u1"}[dtype]
    return torch.as_tensor(_CudaArray(ptr, shape, ts), device=device)


def _ptr(t: torch.Tensor) -> int:
    return t.data_ptr()


def _stamp(t):
    """Identity of a field's contents: storage address, in-place version,
    shape and device of a tensor (None for other arrays)."""
    if isinstance(t, torch.Tensor):
        return (t.data_ptr(), t._version, tuple(t.shape), str(t.device), t.dtype)
    return None


class Device:
    """One data-parallel rendering device (all logical ranks on one GPU)."""

    def __init__(self, num_ranks: int, cuda_device: int = 0, stream: Optional[torch.cuda.Stream] = None):
        lib = load()
        self.num_ranks = num_ranks
        self.cuda_device = cuda_device
        self.torch_device = torch.device("cuda", cuda_device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.torch_device)
        h = C.c_void_p()
        _check(lib.dpvCreateDevice(num_ranks, cuda_device, C.c_void_p(self.stream.cuda_stream), C.byref(h)))
        self._h = h
        self.dims = None
        self.ncam = 0
        self.width = self.height = 0
        self.ntf = 0
        self._keep = []
        self._committed = None

    # -- lifecycle ---------------------------------------------------------
    def release(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _check(load().dpvRelease(self._h))
            self._h = None

    def __del__(self):
        try:
            self.release()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.release()

    # -- scene -------------------------------------------------------------
    def set_geometry(self, dims: Sequence[int], origin=(0.0, 0.0, 0.0), spacing: Optional[float] = None):
        sp = 1.0 / (max(dims) - 1) if spacing is None else spacing
        d = (C.c_int * 3)(*[int(x) for x in dims])
        o = (C.c_float * 3)(*[float(x) for x in origin])
        _check(load().dpvSetVolumeGeometry(self._h, d, o, float(sp)))
        self.dims = tuple(int(x) for x in dims)
        self._committed = None        # a new grid discards every brick

    def commit_brick(self, rank: int, lo: Sequence[int], hi: Sequence[int], data, storage: str = "f32",
                     scale: float = 0.0, data_lo: Sequence[int] = (0, 0, 0)):
        """Commit rank's brick from a field box `data` ((nz, ny, nx) tensor or
        array, x fastest) whose first node is data_lo.  float32 data is
        converted to `storage` on the GPU; data already in the storage format
        is copied."""
        st = DTYPES[storage]
        if isinstance(data, np.ndarray):
            arr = np.ascontiguousarray(data)
            on_dev = 0
            ptr = arr.ctypes.data
            src = 0 if arr.dtype == np.float32 else st
            shape = arr.shape
            keep = arr
        else:
            t = data.contiguous()
            on_dev = 1 if t.is_cuda else 0
            ptr = t.data_ptr()
            src = 0 if t.dtype == torch.float32 else st
            if src != 0 and t.dtype != TORCH_STORAGE[st]:
                raise TypeError("data must be float32 or %s" % TORCH_STORAGE[st])
            shape = tuple(t.shape)
            keep = t
        self._committed = None        # no longer the bricks of one known field
        desc = BrickDesc((C.c_int * 3)(*[int(x) for x in lo]), (C.c_int * 3)(*[int(x) for x in hi]), st,
                         float(scale), src, ptr, (C.c_int * 3)(*[int(x) for x in data_lo]),
                         (C.c_int * 3)(int(shape[2]), int(shape[1]), int(shape[0])), on_dev)
        _check(load().dpvCommitBrick(self._h, int(rank), C.byref(desc)))
        self._storage = st
        del keep

    def commit_partition(self, field, partition, storage: str = "f32", scale: float = 0.0):
        """Commit every rank's brick out of one global field.  The device
        remembers which tensor (and which in-place version of it) the bricks
        came from, so that render() can tell whether a volume it is handed
        is still what the bricks hold."""
        for k in range(partition.num_ranks):
            self.commit_brick(k, partition.lo[k], partition.hi[k], field, storage, scale)
        self._committed = (partition, storage, scale, _stamp(field))

    def ensure_volume(self, volume: torch.Tensor) -> bool:
        """Make the committed bricks those of `volume`: if the bricks were
        committed from another tensor, or from this one before an in-place
        change, commit `volume` again with the same partition, storage and
        scale.  Returns True when it re-committed.  Raises if the bricks were
        not committed from one field by commit_partition (the device cannot
        know which field they are)."""
        c = getattr(self, "_committed", None)
        if c is None:
            raise ValueError("the bricks were not committed from one field with commit_partition: the device "
                             "cannot tie them to `volume`")
        if c[3] == _stamp(volume):
            return False
        self.commit_partition(volume.detach(), c[0], c[1], c[2])
        return True

    def set_tf(self, table, vmin: float = 0.0, vmax: float = 1.0):
        if isinstance(table, np.ndarray):
            t = np.ascontiguousarray(table, dtype=np.float32)
            _check(load().dpvSetTransferFunction(self._h, t.ctypes.data, t.shape[0], vmin, vmax, 0))
            n = t.shape[0]
        else:
            t = table.detach().to(torch.float32).contiguous()
            _check(load().dpvSetTransferFunction(self._h, t.data_ptr(), t.shape[0], vmin, vmax, 1 if t.is_cuda else 0))
            n = t.shape[0]
        self.ntf = n
        self.vmin, self.vmax = vmin, vmax
        self._tf_keep = t

    def set_light(self, direction, step_voxels: float = 1.0, ambient: float = 0.25):
        """Directional light of DPV_FRAME_SHADOW: direction toward the light,
        shadow sample spacing in voxels, ambient term k_a."""
        d = (C.c_float * 3)(*[float(x) for x in direction])
        _check(load().dpvSetLight(self._h, d, float(step_voxels), float(ambient)))

    def set_cameras(self, cams: Iterable):
        cams = list(cams)
        arr = (CameraDesc * len(cams))()
        for i, c in enumerate(cams):
            arr[i] = CameraDesc((C.c_float * 3)(*c.eye), (C.c_float * 3)(*c.center), (C.c_float * 3)(*c.up),
                                float(c.fovy_deg))
        _check(load().dpvSetCameras(self._h, arr, len(cams)))
        self.ncam = len(cams)

    def set_frame(self, width: int, height: int, step_voxels: float = 0.5, sigma_max: float = 8.0, ert: float = 0.0,
                  tile=(0, 0), order: bool = False, staged: bool = False, gather: str = "auto",
                  persistent: bool = False, graph: bool = False, iso: Optional[float] = None,
                  ordered: bool = False, skip: bool = False, deep: bool = False, shadow: bool = False):
        """gather: "auto" (cell layout where it fits in half of the free
        device memory, else quad), "cell", "quad" or "linear".  iso: render
        iso-surface fragments at that level instead of volume rendering
        (DPV_FRAME_ISO).  ordered: visibility-ordered march with global early
        termination (DPV_FRAME_ORDERED).  skip: empty-space skipping
        (DPV_FRAME_SKIP).  deep: deep fragments (DPV_FRAME_DEEP: skipping
        splits a brick's segment into up to DEEP_MAX fragments).  shadow:
        volumetric shadows by ray forwarding (DPV_FRAME_SHADOW; set_light
        first)."""
        if gather not in GATHER_FLAGS:
            raise ValueError("gather must be one of %s" % sorted(GATHER_FLAGS))
        flags = (FRAME_ORDER if order else 0) | (FRAME_STAGED if staged else 0) | GATHER_FLAGS[gather] | (
            FRAME_PERSISTENT if persistent else 0) | (FRAME_GRAPH if graph else 0) | (
            FRAME_ISO if iso is not None else 0) | (FRAME_ORDERED if ordered else 0) | (FRAME_SKIP if skip else 0) | (
            FRAME_DEEP if deep else 0) | (FRAME_SHADOW if shadow else 0)
        f = FrameDesc(int(width), int(height), float(step_voxels), float(sigma_max), float(ert), int(tile[0]),
                      int(tile[1]), flags, float(iso) if iso is not None else 0.0)
        _check(load().dpvSetFrame(self._h, C.byref(f)))
        self._frame_args = (step_voxels, sigma_max, ert)
        self._frame_kw = {"order": order, "staged": staged, "graph": graph, "iso": iso, "ordered": ordered,
                          "skip": skip, "deep": deep, "shadow": shadow}
        self.width, self.height = int(width), int(height)

    # -- rendering ---------------------------------------------------------
    def render(self):
        _check(load().dpvRenderFrame(self._h))

    def ready(self, wait: bool = True) -> bool:
        r = C.c_int()
        _check(load().dpvFrameReady(self._h, 1 if wait else 0, C.byref(r)))
        return bool(r.value)

    def map_frame(self, camera: int = 0):
        """Zero-copy views (valid until the next render): rgba (H, W, 4), depth (H, W)."""
        r, d = C.c_void_p(), C.c_void_p()
        _check(load().dpvMapFrame(self._h, camera, C.byref(r), C.byref(d)))
        rgba = _wrap(r.value, (self.height, self.width, 4), torch.float32, self.torch_device)
        depth = _wrap(d.value, (self.height, self.width), torch.float32, self.torch_device)
        return rgba, depth

    def frames(self):
        """All cameras' frames as zero-copy views: (ncam, H, W, 4), (ncam, H, W)."""
        r, d = C.c_void_p(), C.c_void_p()
        _check(load().dpvMapFrame(self._h, 0, C.byref(r), C.byref(d)))
        rgba = _wrap(r.value, (self.ncam, self.height, self.width, 4), torch.float32, self.torch_device)
        depth = _wrap(d.value, (self.ncam, self.height, self.width), torch.float32, self.torch_device)
        return rgba, depth

    def copy_frame(self, camera: int, rgba: Optional[torch.Tensor], depth: Optional[torch.Tensor] = None):
        _check(load().dpvCopyFrame(self._h, camera, _ptr(rgba) if rgba is not None else None,
                                   _ptr(depth) if depth is not None else None))

    def copy_frame_async(self, camera: int, rgba: Optional[torch.Tensor], depth: Optional[torch.Tensor] = None):
        """Issue the copy of camera's frame (camera -1: all cameras) and
        return; the destination is complete after copy_wait().  It runs on a
        copy stream beside the next render (pinned host memory overlaps)."""
        _check(load().dpvCopyFrameAsync(self._h, camera, _ptr(rgba) if rgba is not None else None,
                                        _ptr(depth) if depth is not None else None))

    def copy_wait(self):
        _check(load().dpvCopyWait(self._h))

    def map_fragments(self, camera: int, rank: int):
        """Zero-copy views of rank's fragments of one camera (dpvMapFragments):
        rgba (H, W, 4) premultiplied and key (H, W) int32 (KEY_EMPTY = none),
        valid until unmap_fragments(camera, rank) or release."""
        p = C.c_void_p()
        _check(load().dpvMapFragments(self._h, camera, rank, C.byref(p)))
        npix = self.height * self.width
        rgba = _wrap(p.value, (self.height, self.width, 4), torch.float32, self.torch_device)
        key = _wrap(p.value + 16 * npix, (self.height, self.width), torch.int32, self.torch_device)
        return rgba, key

    def unmap_fragments(self, camera: int, rank: int):
        _check(load().dpvUnmapFragments(self._h, camera, rank))

    def read_fragments(self, camera: int, rank: int, layer: int = 0):
        """Rank's fragments of one camera (fragment layer `layer` of a deep frame)."""
        rgba = torch.empty((self.height, self.width, 4), dtype=torch.float32, device=self.torch_device)
        key = torch.empty((self.height, self.width), dtype=torch.int32, device=self.torch_device)
        _check(load().dpvReadDeepFragments(self._h, camera, rank, layer, _ptr(rgba), _ptr(key)))
        return rgba, key

    def read_brick(self, rank: int):
        """(stored nodes (nz, ny, nx) in the storage dtype, first stored node, scale)."""
        lo, n, sc = (C.c_int * 3)(), (C.c_int * 3)(), C.c_float()
        _check(load().dpvReadBrick(self._h, rank, None, lo, n, C.byref(sc)))
        dt = TORCH_STORAGE[self._storage]
        out = torch.empty((n[2], n[1], n[0]), dtype=dt, device=self.torch_device)
        _check(load().dpvReadBrick(self._h, rank, _ptr(out), lo, n, C.byref(sc)))
        return out, tuple(lo), sc.value

    def order(self, camera: int = 0) -> torch.Tensor:
        p, s = C.c_void_p(), C.c_int()
        _check(load().dpvMapOrder(self._h, camera, C.byref(p), C.byref(s)))
        return _wrap(p.value, (self.height, self.width, s.value), torch.uint8, self.torch_device)

    def backward(self, grad_rgba: torch.Tensor, volume_grad: bool = True):
        """Adjoint of the last render: returns (dL/dTF (n, 4) float64, dL/dfield (nz, ny, nx) float32 or None)."""
        g = grad_rgba.to(torch.float32).contiguous()
        if g.numel() != self.ncam * self.height * self.width * 4:
            raise ValueError("grad_rgba must have %d x %d x %d x 4 elements" % (self.ncam, self.height, self.width))
        dtf = torch.empty((self.ntf, 4), dtype=torch.float64, device=self.torch_device)
        dvol = None
        if volume_grad:
            dvol = torch.empty((self.dims[2], self.dims[1], self.dims[0]), dtype=torch.float32, device=self.torch_device)
        _check(load().dpvBackward(self._h, _ptr(g), _ptr(dtf), _ptr(dvol) if dvol is not None else None))
        self._grad_keep = g
        return dtf, dvol

    def stats(self) -> dict:
        s = Stats()
        _check(load().dpvGetStats(self._h, C.byref(s)))
        out = {k: getattr(s, k) for k, _ in Stats._fields_ if k not in ("stage_ms", "stage_calls")}
        out["stage_ms"] = {n: s.stage_ms[i] for i, n in enumerate(STAGES)}
        out["stage_calls"] = {n: s.stage_calls[i] for i, n in enumerate(STAGES)}
        return out

    def autotune(self, frames: int = 3, cache: Optional[str] = None, key: Optional[str] = None) -> dict:
        """Pick the fastest tile shape / gather layout / schedule for the
        current scene (dpvAutotune).  With `cache` (a JSON file) and `key`, a
        stored choice for this key and GPU is applied instead of re-timing,
        and new choices are stored."""
        import json
        gpu = torch.cuda.get_device_name(self.cuda_device)
        entry = None
        if cache and key and os.path.exists(cache):
            with open(cache) as f:
                entry = json.load(f).get(gpu, {}).get(key)
        if entry:
            self._tune_apply(entry)
            return dict(entry, cached=True)
        r = TuneResult()
        _check(load().dpvAutotune(self._h, int(frames), C.byref(r)))
        res = {"tile": [r.tile_w, r.tile_h], "flags": r.flags, "ms": r.ms, "candidates": r.candidates}
        self._tuned = res
        if cache and key:
            data = {}
            if os.path.exists(cache):
                with open(cache) as f:
                    data = json.load(f)
            data.setdefault(gpu, {})[key] = res
            with open(cache, "w") as f:
                json.dump(data, f, indent=1)
        return dict(res, cached=False)

    def _tune_apply(self, entry):
        fl = entry["flags"]
        self.set_frame(self.width, self.height, *self._frame_args, tile=tuple(entry["tile"]),
                       gather=gather_of(fl), persistent=bool(fl & FRAME_PERSISTENT), **self._frame_kw)

    def reset_stats(self):
        _check(load().dpvResetStats(self._h))

    def set_profiling(self, on: bool = True):
        _check(load().dpvSetProfiling(self._h, 1 if on else 0))


def render_noalloc(dims: Sequence[int], bricks, storage: str, tf: torch.Tensor, camera, width: int, height: int,
                   rgba: torch.Tensor, depth: torch.Tensor, step_voxels: float = 0.5, sigma_max: float = 8.0,
                   ert: float = 0.0, tile=(0, 0), vmin: float = 0.0, vmax: float = 1.0, origin=(0.0, 0.0, 0.0),
                   spacing: Optional[float] = None, stream: Optional[torch.cuda.Stream] = None, flags: int = 0):
    """Allocation-free render of one camera (dpvRenderNoAlloc) into caller
    tensors rgba (H, W, 4) and depth (H, W) on the current CUDA device.
    bricks: per rank (owned_lo, owned_hi, stored nodes as a device tensor in
    the storage dtype, scale).  Nothing is allocated on the device; see
    include/dpv.h for the size limit and the rule that calls must not overlap
    on the GPU.  flags: DPV_FRAME_* bits (the iso, ordered and skip bits
    are refused; the layout bits are ignored)."""
    sp = 1.0 / (max(dims) - 1) if spacing is None else spacing
    arr = (NoAllocBrick * len(bricks))()
    for i, (lo, hi, data, scale) in enumerate(bricks):
        arr[i] = NoAllocBrick((C.c_int * 3)(*[int(x) for x in lo]), (C.c_int * 3)(*[int(x) for x in hi]),
                              data.data_ptr(), float(scale))
    t = tf.detach().to(torch.float32).contiguous()
    sc = NoAllocScene((C.c_int * 3)(*[int(x) for x in dims]), (C.c_float * 3)(*[float(x) for x in origin]), float(sp),
                      len(bricks), arr, DTYPES[storage], t.data_ptr(), t.shape[0], float(vmin), float(vmax))
    cam = CameraDesc((C.c_float * 3)(*camera.eye), (C.c_float * 3)(*camera.center), (C.c_float * 3)(*camera.up),
                     float(camera.fovy_deg))
    fr = FrameDesc(int(width), int(height), float(step_voxels), float(sigma_max), float(ert), int(tile[0]),
                   int(tile[1]), int(flags), 0.0)
    st = stream if stream is not None else torch.cuda.current_stream()
    _check(load().dpvRenderNoAlloc(C.byref(sc), C.byref(cam), C.byref(fr), _ptr(rgba), _ptr(depth),
                                   C.c_void_p(st.cuda_stream)))


class RenderFunction(torch.autograd.Function):
    """Differentiable render: images of all cameras as a function of the TF
    table and (for the gradient) the global field `volume`.  The forward
    uploads `tf`, makes the committed bricks those of `volume` (committing
    it again if the bricks came from another tensor or from an older
    in-place version of this one), and renders; the backward runs the
    library's adjoint (compositor + ray-march replay), whose field gradient
    is then the gradient for `volume` as it was at the forward."""

    @staticmethod
    def forward(ctx, tf: torch.Tensor, volume: Optional[torch.Tensor], device: Device, vmin: float, vmax: float):
        if volume is not None:
            device.ensure_volume(volume)
        device.set_tf(tf, vmin, vmax)
        device.render()
        rgba, _ = device.frames()
        ctx.device = device
        ctx.want_volume = volume is not None and volume.requires_grad
        ctx.tf_dtype = tf.dtype
        return rgba.clone()

    @staticmethod
    def backward(ctx, g):
        dtf, dvol = ctx.device.backward(g, volume_grad=ctx.want_volume)
        return dtf.to(ctx.tf_dtype), dvol, None, None, None


DPVRender = RenderFunction


def render(device: Device, tf: torch.Tensor, volume: Optional[torch.Tensor] = None, vmin: float = 0.0,
           vmax: float = 1.0) -> torch.Tensor:
    """(ncam, H, W, 4) premultiplied RGBA, differentiable in tf (and volume)."""
    return RenderFunction.apply(tf, volume, device, vmin, vmax)
