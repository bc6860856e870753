"""FP64 CPU oracle for the data-parallel volume rendering path.

TEST INFRASTRUCTURE ONLY: imported by the tests, by the smoke check and by the
benchmark's CPU-baseline leg, never by the product package.  The C source
(`dpv_oracle.c`) is compiled with gcc into `liboracle.so` next to it on first
use (or by `build()`); it shares no code with the CUDA path.

Each wrapper states the passage or reading it follows; the arithmetic itself
is in the C file.
"""
from __future__ import annotations

import contextlib
import ctypes as C
import os
import subprocess
from dataclasses import dataclass
from typing import List, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dpv_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

F32, F16, BF16, FP8 = 0, 1, 2, 3
DTYPE_NAMES = {"f32": F32, "f16": F16, "bf16": BF16, "fp8": FP8}
NP_STORAGE = {F32: np.float32, F16: np.uint16, BF16: np.uint16, FP8: np.uint8}
KEY_EMPTY = 2 ** 31 - 1
FLAG_HIT, FLAG_EXIT_AMBIG, FLAG_OWNER_AMBIG, FLAG_ERT_AMBIG = 1, 2, 4, 8
FLAG_ISO_AMBIG = 16
FLAG_MACRO_AMBIG = 32
FLAG_SHADOW_AMBIG = 64
ISO_EPS = 5e-5   # iso ambiguity band on s (a rounded sample may cross otherwise)


_CFLAGS = ["-O2", "-std=c11", "-D_GNU_SOURCE", "-fopenmp", "-fPIC", "-shared", "-fno-fast-math",
           "-ffp-contract=off"]


def compile_source(src: str, out: str) -> str:
    """Compile an oracle C source (gcc, the flags of build()) into `out`."""
    tmp = out + ".tmp.%d" % os.getpid()
    subprocess.check_call(["gcc", *_CFLAGS, "-o", tmp, src, "-lm"])
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile the oracle (gcc, -O2, OpenMP) if missing or stale."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        compile_source(_SRC, _LIB)
    return _LIB


class _Grid(C.Structure):
    _fields_ = [("dims", C.c_int * 3), ("origin", C.c_double * 3), ("spacing", C.c_double)]


class _Camera(C.Structure):
    _fields_ = [("eye", C.c_double * 3), ("center", C.c_double * 3), ("up", C.c_double * 3),
                ("fovy_deg", C.c_double)]


class _Frame(C.Structure):
    _fields_ = [("width", C.c_int), ("height", C.c_int), ("step_voxels", C.c_double),
                ("sigma_max", C.c_double), ("ert", C.c_double), ("amb_samples", C.c_double),
                ("amb_alpha", C.c_double)]


class _Brick(C.Structure):
    _fields_ = [("owned_lo", C.c_int * 3), ("owned_hi", C.c_int * 3), ("dtype", C.c_int),
                ("scale", C.c_double), ("data", C.c_void_p)]


class _Light(C.Structure):
    _fields_ = [("dir", C.c_double * 3), ("step_voxels", C.c_double), ("ambient", C.c_double)]


class _TF(C.Structure):
    _fields_ = [("rgba", C.c_void_p), ("n", C.c_int), ("vmin", C.c_double), ("vmax", C.c_double)]


_lib = None


def _configure(l):
    P = C.c_void_p
    l.orc_render_full.argtypes = [P, P, P, P, P, C.c_int, P, P, P, P]
    l.orc_render_bricks.argtypes = [P, C.c_int, P, P, P, P, C.c_int, P, P, P, P, P, P, P, P, P, P]
    l.orc_grad_bricks.argtypes = [P, C.c_int, P, P, P, P, C.c_int, P, P, P, P, P, C.c_double, P]
    l.orc_composite.argtypes = [C.c_int, C.c_int, P, P, P, P]
    l.orc_render_ordered.argtypes = [P, P, C.c_int, P, P, P, P, C.c_int, P, P, P, P, P, P]
    l.orc_render_iso.argtypes = [P, P, C.c_int, P, P, P, P, C.c_double, C.c_double, C.c_int, P, P, P, P, P,
                                 P, P]
    l.orc_render_deep.argtypes = [P, C.c_int, P, P, P, P, C.c_int, C.c_int, P, P, P, P, P, P, P, P]
    l.orc_render_shadow.argtypes = [P, P, C.c_int, P, P, P, P, P, C.c_int, P, P, P, P, P, P]
    l.orc_light_transmittance.argtypes = [P, P, C.c_int, P, P, P, P, C.c_int, P, P, P, P]
    l.orc_kd_order.argtypes = [C.c_int, P, P, P, P, P, P]
    l.orc_kd_order.restype = C.c_int
    l.orc_camera_ray.argtypes = [P, C.c_int, C.c_int, C.c_int, C.c_int, P, P]
    l.orc_brick_scale.argtypes = [P, C.c_int64, C.c_int]
    l.orc_brick_scale.restype = C.c_float
    l.orc_quantize.argtypes = [P, C.c_int64, C.c_int, C.c_float, P]
    l.orc_dequantize.argtypes = [P, C.c_int64, C.c_int, C.c_double, P]
    l.orc_stored_box.argtypes = [P, P, P, P, P]
    l.orc_extract_brick.argtypes = [P, P, P, P, P]
    l.orc_max_threads.restype = C.c_int
    l.orc_set_threads.argtypes = [C.c_int]
    return l


def lib():
    global _lib
    if _lib is None:
        _lib = _configure(C.CDLL(build()))
    return _lib


@contextlib.contextmanager
def library(path: str):
    """Run every wrapper against another build of an oracle source (the
    tests compile copies with a planted mistake to show that a pin fails)."""
    global _lib
    prev = lib()
    _lib = _configure(C.CDLL(path))
    try:
        yield _lib
    finally:
        _lib = prev


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))


def max_threads() -> int:
    return int(lib().orc_max_threads())


@dataclass
class Frame:
    """Frame parameters: image size, step in voxels, sigma_max,
    per-fragment early-termination threshold (0 = off) and the ambiguity
    bands used for flags."""
    width: int
    height: int
    step_voxels: float = 0.5
    sigma_max: float = 8.0
    ert: float = 0.0
    amb_samples: float = 1e-2
    amb_alpha: float = 1e-4

    def c(self) -> _Frame:
        return _Frame(self.width, self.height, self.step_voxels, self.sigma_max, self.ert,
                      self.amb_samples, self.amb_alpha)


def _grid(dims, origin=(0.0, 0.0, 0.0), spacing=None) -> _Grid:
    sp = 1.0 / (max(dims) - 1) if spacing is None else spacing
    return _Grid((C.c_int * 3)(*dims), (C.c_double * 3)(*origin), sp)


def _camera(cam) -> _Camera:
    return _Camera((C.c_double * 3)(*cam.eye), (C.c_double * 3)(*cam.center), (C.c_double * 3)(*cam.up),
                   float(cam.fovy_deg))


def _tf(tab: np.ndarray, vmin: float, vmax: float):
    tab = np.ascontiguousarray(tab, dtype=np.float32)
    return _TF(tab.ctypes.data, tab.shape[0], vmin, vmax), tab


def _pix(pix, frame: Frame):
    if pix is None:
        return frame.width * frame.height, None, None
    arr = np.ascontiguousarray(pix, dtype=np.int32)
    return int(arr.size), _p(arr), arr


# ---------------------------------------------------------------------------
# number formats and bricks (brick commit)
# ---------------------------------------------------------------------------

def brick_scale(values: np.ndarray, dtype: int) -> np.float32:
    v = np.ascontiguousarray(values, dtype=np.float32)
    return np.float32(lib().orc_brick_scale(_p(v), v.size, dtype))


def quantize(values: np.ndarray, dtype: int, scale: float = 1.0) -> np.ndarray:
    v = np.ascontiguousarray(values, dtype=np.float32)
    out = np.empty(v.shape, dtype=NP_STORAGE[dtype])
    lib().orc_quantize(_p(v), v.size, dtype, float(np.float32(scale)), _p(out))
    return out


def dequantize(stored: np.ndarray, dtype: int, scale: float = 1.0) -> np.ndarray:
    s = np.ascontiguousarray(stored)
    out = np.empty(s.shape, dtype=np.float64)
    lib().orc_dequantize(_p(s), s.size, dtype, float(scale), _p(out))
    return out


def stored_box(dims, lo, hi):
    """(first node, node count) per axis of the nodes a rank stores."""
    d = np.array(dims, np.int32)
    l = np.array(lo, np.int32)
    h = np.array(hi, np.int32)
    s_lo = np.zeros(3, np.int32)
    s_n = np.zeros(3, np.int32)
    lib().orc_stored_box(_p(d), _p(l), _p(h), _p(s_lo), _p(s_n))
    return s_lo, s_n


def extract_brick(field: np.ndarray, lo, hi) -> np.ndarray:
    f = np.ascontiguousarray(field, dtype=np.float32)
    dims = np.array([f.shape[2], f.shape[1], f.shape[0]], np.int32)
    _, s_n = stored_box(dims, lo, hi)
    out = np.empty((s_n[2], s_n[1], s_n[0]), np.float32)
    l = np.array(lo, np.int32)
    h = np.array(hi, np.int32)
    lib().orc_extract_brick(_p(f), _p(dims), _p(l), _p(h), _p(out))
    return out


@dataclass
class Brick:
    lo: Sequence[int]
    hi: Sequence[int]
    dtype: int
    scale: float
    data: np.ndarray          # stored nodes in the storage format


def make_bricks(field: np.ndarray, partition, dtype: int = F32) -> List[Brick]:
    """The oracle's own brick commit: extract stored nodes (owned + 1 ghost),
    choose the per-brick scale and quantise."""
    out = []
    for k in range(partition.num_ranks):
        lo, hi = [int(x) for x in partition.lo[k]], [int(x) for x in partition.hi[k]]
        v = extract_brick(field, lo, hi)
        sc = brick_scale(v, dtype)
        out.append(Brick(lo, hi, dtype, float(sc), quantize(v, dtype, sc)))
    return out


def _bricks_c(bricks: List[Brick]):
    arr = (_Brick * len(bricks))()
    keep = []
    for i, b in enumerate(bricks):
        d = np.ascontiguousarray(b.data)
        keep.append(d)
        arr[i] = _Brick((C.c_int * 3)(*b.lo), (C.c_int * 3)(*b.hi), b.dtype, float(b.scale), d.ctypes.data)
    return arr, keep


# ---------------------------------------------------------------------------
# rendering
# ---------------------------------------------------------------------------

def camera_ray(cam, width: int, height: int, px: int, py: int):
    """Eye and unit direction of the ray through pixel (px, py)."""
    o = np.zeros(3)
    d = np.zeros(3)
    c = _camera(cam)
    lib().orc_camera_ray(C.byref(c), width, height, px, py, _p(o), _p(d))
    return o, d


def render_full(field: np.ndarray, tf: np.ndarray, cam, frame: Frame, pix=None, vmin=0.0, vmax=1.0,
                origin=(0.0, 0.0, 0.0), spacing=None):
    """Unpartitioned FP64 render of the global float32 field (no early
    termination): the plain definition the partitioned path reproduces."""
    f = np.ascontiguousarray(field, dtype=np.float32)
    dims = (f.shape[2], f.shape[1], f.shape[0])
    g = _grid(dims, origin, spacing)
    t, tab = _tf(tf, vmin, vmax)
    cam_c = _camera(cam)
    fr = frame.c()
    n, pp, keep = _pix(pix, frame)
    rgba = np.zeros((n, 4))
    ns = np.zeros(n, np.int64)
    fl = np.zeros(n, np.uint8)
    lib().orc_render_full(C.byref(g), _p(f), C.byref(t), C.byref(cam_c), C.byref(fr), n, pp, _p(rgba), _p(ns), _p(fl))
    return {"rgba": rgba, "nsamples": ns, "flags": fl}


def render_bricks(dims, bricks: List[Brick], tf: np.ndarray, cam, frame: Frame, pix=None, vmin=0.0, vmax=1.0,
                  origin=(0.0, 0.0, 0.0), spacing=None):
    """Partitioned FP64 render: per-brick fragments (with per-fragment early
    termination when frame.ert is set), sort by key, front-to-back over."""
    g = _grid(dims, origin, spacing)
    t, tab = _tf(tf, vmin, vmax)
    cam_c = _camera(cam)
    fr = frame.c()
    K = len(bricks)
    barr, keep_b = _bricks_c(bricks)
    n, pp, keep = _pix(pix, frame)
    res = {
        "rgba": np.zeros((n, 4)), "depth": np.zeros(n), "order": np.zeros((n, K), np.uint8),
        "frag_rgba": np.zeros((n, K, 4)), "frag_key": np.zeros((n, K), np.int32),
        "frag_nsamp": np.zeros((n, K), np.int32), "frag_margin": np.zeros((n, K)),
        "nsamples": np.zeros(n, np.int64), "flags": np.zeros(n, np.uint8),
    }
    lib().orc_render_bricks(C.byref(g), K, barr, C.byref(t), C.byref(cam_c), C.byref(fr), n, pp,
                            _p(res["rgba"]), _p(res["depth"]), _p(res["order"]), _p(res["frag_rgba"]),
                            _p(res["frag_key"]), _p(res["frag_nsamp"]), _p(res["frag_margin"]),
                            _p(res["nsamples"]), _p(res["flags"]))
    return res


def render_deep(dims, bricks: List[Brick], tf: np.ndarray, cam, frame: Frame, deep: int = 4, pix=None, vmin=0.0,
                vmax=1.0, origin=(0.0, 0.0, 0.0), spacing=None):
    """FP64 deep-fragment render: empty-space skipping over macro-cells of
    8^3 cells splits each brick's segment into one fragment per run of
    evaluated samples (at most `deep` per brick; later runs continue the
    last), every fragment of the pixel sorted by key and blended front to
    back.  Returns rgba, depth, frag_rgba (n, K, deep, 4), frag_key
    (n, K, deep; 2^31 - 1 = none), frag_count (n, K), nsamples (evaluated)
    and flags (FLAG_MACRO_AMBIG among them)."""
    g = _grid(dims, origin, spacing)
    t, tab = _tf(tf, vmin, vmax)
    cam_c = _camera(cam)
    fr = frame.c()
    K = len(bricks)
    barr, keep_b = _bricks_c(bricks)
    n, pp, keep = _pix(pix, frame)
    res = {"rgba": np.zeros((n, 4)), "depth": np.zeros(n), "frag_rgba": np.zeros((n, K, deep, 4)),
           "frag_key": np.zeros((n, K, deep), np.int32), "frag_count": np.zeros((n, K), np.int32),
           "nsamples": np.zeros(n, np.int64), "flags": np.zeros(n, np.uint8)}
    lib().orc_render_deep(C.byref(g), K, barr, C.byref(t), C.byref(cam_c), C.byref(fr), int(deep), n, pp,
                          _p(res["rgba"]), _p(res["depth"]), _p(res["frag_rgba"]), _p(res["frag_key"]),
                          _p(res["frag_count"]), _p(res["nsamples"]), _p(res["flags"]))
    return res


@dataclass
class Light:
    """Directional light: unit direction toward the light, shadow sample
    spacing h in node units, ambient term k_a."""
    direction: tuple = (0.0, 0.0, 1.0)
    step_voxels: float = 1.0
    ambient: float = 0.25

    def c(self) -> _Light:
        d = np.asarray(self.direction, np.float64)
        d = d / np.linalg.norm(d)
        return _Light((C.c_double * 3)(*d), self.step_voxels, self.ambient)


def _source(dims, field, bricks):
    if (field is None) == (bricks is None):
        raise ValueError("give exactly one of field and bricks")
    if bricks is not None:
        barr, keep = _bricks_c(bricks)
        return None, len(bricks), barr, keep
    f = np.ascontiguousarray(field, dtype=np.float32)
    assert f.shape == (dims[2], dims[1], dims[0])
    return _p(f), 1, None, f


def render_shadow(dims, tf: np.ndarray, cam, frame: Frame, light: Light, field=None, bricks=None, pix=None,
                  vmin=0.0, vmax=1.0, origin=(0.0, 0.0, 0.0), spacing=None):
    """FP64 shadowed render: each sample's emission scaled by
    k_a + (1 - k_a) T_light, T_light the transmittance of its shadow ray
    toward the directional light.  With `field` the plain definition (no
    early termination); with `bricks` per-brick fragments (frame.ert per
    fragment), shadow samples evaluated by their owner bricks, sort-last
    composite.  Returns rgba, depth, nsamples, nshadow and flags."""
    g = _grid(dims, origin, spacing)
    t, tab = _tf(tf, vmin, vmax)
    cam_c = _camera(cam)
    fr = frame.c()
    lc = light.c()
    f_ptr, K, barr, keep_s = _source(dims, field, bricks)
    n, pp, keep = _pix(pix, frame)
    res = {"rgba": np.zeros((n, 4)), "depth": np.zeros(n), "nsamples": np.zeros(n, np.int64),
           "nshadow": np.zeros(n, np.int64), "flags": np.zeros(n, np.uint8)}
    lib().orc_render_shadow(C.byref(g), f_ptr, K, barr, C.byref(t), C.byref(cam_c), C.byref(fr), C.byref(lc), n, pp,
                            _p(res["rgba"]), _p(res["depth"]), _p(res["nsamples"]), _p(res["nshadow"]),
                            _p(res["flags"]))
    return res


def light_transmittance(dims, tf: np.ndarray, points: np.ndarray, light: Light, sigma_max: float = 8.0,
                        field=None, bricks=None, vmin=0.0, vmax=1.0, origin=(0.0, 0.0, 0.0), spacing=None):
    """T_light at node-space points (n, 3); also the shadow sample counts and
    the face-ambiguity flags."""
    g = _grid(dims, origin, spacing)
    t, tab = _tf(tf, vmin, vmax)
    fr = Frame(1, 1, sigma_max=sigma_max).c()
    lc = light.c()
    f_ptr, K, barr, keep_s = _source(dims, field, bricks)
    pts = np.ascontiguousarray(points, dtype=np.float64).reshape(-1, 3)
    T = np.zeros(len(pts))
    cnt = np.zeros(len(pts), np.int64)
    amb = np.zeros(len(pts), np.uint8)
    lib().orc_light_transmittance(C.byref(g), f_ptr, K, barr, C.byref(t), C.byref(fr), C.byref(lc), len(pts),
                                  _p(pts), _p(T), _p(cnt), _p(amb))
    return T, cnt, amb


def render_ordered(dims, tf: np.ndarray, cam, frame: Frame, field=None, bricks=None, pix=None, vmin=0.0, vmax=1.0,
                   origin=(0.0, 0.0, 0.0), spacing=None):
    """FP64 visibility-ordered march with global early termination
    (frame.ert on the accumulated opacity; 0 = off): with `field` the
    unpartitioned plain definition, with `bricks` each sample evaluated by
    its owning brick, bricks in ray order carrying the transmittance.
    Returns rgba, depth, depth_alpha (opacity the depth's segment adds),
    nsamples (evaluated) and flags."""
    if (field is None) == (bricks is None):
        raise ValueError("give exactly one of field and bricks")
    g = _grid(dims, origin, spacing)
    t, tab = _tf(tf, vmin, vmax)
    cam_c = _camera(cam)
    fr = frame.c()
    n, pp, keep = _pix(pix, frame)
    res = {"rgba": np.zeros((n, 4)), "depth": np.zeros(n), "depth_alpha": np.zeros(n),
           "nsamples": np.zeros(n, np.int64), "flags": np.zeros(n, np.uint8)}
    if bricks is not None:
        barr, keep_b = _bricks_c(bricks)
        f_ptr, K = None, len(bricks)
    else:
        f = np.ascontiguousarray(field, dtype=np.float32)
        assert f.shape == (dims[2], dims[1], dims[0])
        barr, f_ptr, K = None, _p(f), 1
    lib().orc_render_ordered(C.byref(g), f_ptr, K, barr, C.byref(t), C.byref(cam_c), C.byref(fr), n, pp,
                             _p(res["rgba"]), _p(res["depth"]), _p(res["depth_alpha"]), _p(res["nsamples"]),
                             _p(res["flags"]))
    return res


def render_iso(dims, tf: np.ndarray, cam, frame: Frame, iso: float, field=None, bricks=None, pix=None, vmin=0.0,
               vmax=1.0, origin=(0.0, 0.0, 0.0), spacing=None, iso_eps=ISO_EPS):
    """FP64 iso-surface render: the first sample pair of the ray across
    which [s >= iso] changes, the surface point interpolated linearly between
    them, shaded TF rgb(iso) x (0.25 + 0.75 |N.d|/(|N||d|)), opaque.  With
    `field` (nz, ny, nx float32) the plain definition on the whole field;
    with `bricks` each brick finds the first hit among the pairs whose later
    sample it owns, and the depth composite keeps the smallest key.
    Returns rgba, depth (+inf: no hit), key (-1: no hit), dsdt
    (|s_h - s_{h-1}|), frag_key (bricks; 2^31 - 1 = none) and flags."""
    if (field is None) == (bricks is None):
        raise ValueError("give exactly one of field and bricks")
    g = _grid(dims, origin, spacing)
    t, tab = _tf(tf, vmin, vmax)
    cam_c = _camera(cam)
    fr = frame.c()
    n, pp, keep = _pix(pix, frame)
    K = len(bricks) if bricks is not None else 1
    res = {"rgba": np.zeros((n, 4)), "depth": np.zeros(n), "key": np.zeros(n, np.int64), "dsdt": np.zeros(n),
           "frag_key": np.zeros((n, K), np.int32), "flags": np.zeros(n, np.uint8)}
    if bricks is not None:
        barr, keep_b = _bricks_c(bricks)
        f_ptr = None
    else:
        f = np.ascontiguousarray(field, dtype=np.float32)
        assert f.shape == (dims[2], dims[1], dims[0])
        barr, f_ptr = None, _p(f)
    lib().orc_render_iso(C.byref(g), f_ptr, K, barr, C.byref(t), C.byref(cam_c), C.byref(fr), float(iso),
                         float(iso_eps), n, pp, _p(res["rgba"]), _p(res["depth"]), _p(res["key"]), _p(res["dsdt"]),
                         _p(res["frag_key"]) if bricks is not None else None, _p(res["flags"]))
    return res


KNOT_EPS = 4e-3   # knot ambiguity band, in TF entries (u units)


def grad_bricks(dims, bricks: List[Brick], tf: np.ndarray, cam, frame: Frame, grad_rgba: np.ndarray, pix=None,
                vmin=0.0, vmax=1.0, want_volume=True, origin=(0.0, 0.0, 0.0), spacing=None, knot_eps=None,
                tf_amb=False):
    """FP64 reverse-mode gradient of sum(grad_rgba * image) with respect to the
    TF table (n x 4) and the global field (nz, ny, nx).

    With knot_eps (in TF entries, e.g. KNOT_EPS) also returns the knot
    ambiguity of the field gradient (nz, ny, nx): per voxel, how far a
    correct gradient may lie from the returned one because samples within
    knot_eps of a TF knot may take either one-sided slope there.  The lerp's
    derivative jumps at such knots, so an s rounded to the other side of one
    gives the other, equally correct, derivative.

    With tf_amb also returns the TF-coordinate ambiguity of the TF gradient
    (n x 4): per entry, the sum over samples of du |g| with
    du = 2^-22 max(u, 1), how far an FP32 u (about three roundings of
    2^-24 u) may move the split of a sample's value adjoint g between the
    entries i0 and i0 + 1."""
    g = _grid(dims, origin, spacing)
    t, tab = _tf(tf, vmin, vmax)
    cam_c = _camera(cam)
    fr = frame.c()
    K = len(bricks)
    barr, keep_b = _bricks_c(bricks)
    n, pp, keep = _pix(pix, frame)
    gr = np.ascontiguousarray(grad_rgba, dtype=np.float64).reshape(n, 4)
    dtf = np.zeros((tab.shape[0], 4))
    dvol = np.zeros((dims[2], dims[1], dims[0])) if want_volume else None
    damb = np.zeros((dims[2], dims[1], dims[0])) if knot_eps is not None else None
    tamb = np.zeros_like(dtf) if tf_amb else None
    lib().orc_grad_bricks(C.byref(g), K, barr, C.byref(t), C.byref(cam_c), C.byref(fr), n, pp, _p(gr), _p(dtf),
                          _p(dvol) if dvol is not None else None, _p(damb) if damb is not None else None,
                          float(knot_eps or 0.0), _p(tamb) if tamb is not None else None)
    out = (dtf, dvol) + ((damb,) if knot_eps is not None else ()) + ((tamb,) if tf_amb else ())
    return out


def composite(frag_rgba: np.ndarray, frag_key: np.ndarray):
    """Sort-last composite of given fragments (npix, K, 4) / (npix, K)."""
    fr = np.ascontiguousarray(frag_rgba, dtype=np.float64)
    fk = np.ascontiguousarray(frag_key, dtype=np.int32)
    n, K = fk.shape
    rgba = np.zeros((n, 4))
    order = np.zeros((n, K), np.uint8)
    lib().orc_composite(n, K, _p(fr), _p(fk), _p(rgba), _p(order))
    return rgba, order


def kd_order(partition, eye_node) -> np.ndarray:
    """Front-to-back leaf order of the partition's k-d tree from a point given
    in node coordinates."""
    K = partition.num_ranks
    out = np.zeros(K, np.uint8)
    ax = np.ascontiguousarray(partition.axis, np.int32)
    sp = np.ascontiguousarray(partition.split, np.int32)
    le = np.ascontiguousarray(partition.left, np.int32)
    ri = np.ascontiguousarray(partition.right, np.int32)
    e = np.ascontiguousarray(eye_node, np.float64)
    m = lib().orc_kd_order(int(ax.size), _p(ax), _p(sp), _p(le), _p(ri), _p(e), _p(out))
    return out[:m]
