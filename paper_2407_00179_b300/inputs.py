"""Seeded synthetic inputs shared by the CUDA path, the FP64 oracle, the tests
and the benchmark.

This module only *makes inputs*: scalar fields, transfer-function tables,
cameras and brick partitions.  It holds none of the rendering arithmetic (no
rays, no sampling, no compositing), so that the oracle and the CUDA path can
both consume its outputs without sharing any of the method's code.

The paper (§6, figures of the ParaView/VisIt and DNS examples) renders large
simulation volumes (thunderstorm 2501x3001x305, aircraft 1225x580x2000, DNS
10240x7680x1536) split one part per rank (§1, §3.1.2).  Those datasets are not
available, so seeded synthetic fields of the same kind of structure stand in:
smooth Gaussian blobs, multi-octave value noise, and a log-normal,
turbulence-like variant.  All random draws use numpy's PCG64 with a base seed
and a per-object stream id, so every object is reproducible in isolation.

Conventions (fixed here because the inputs depend on them):
  * fields are node-centred, stored x-fastest as tensors of shape (nz, ny, nx);
  * node i of an axis sits at world coordinate ``origin + i * spacing`` with
    ``origin = 0`` and ``spacing = 1 / (max(dims) - 1)``, so the longest axis
    spans [0, 1];
  * a brick partition assigns each rank a half-open node range per axis.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional, Sequence, Tuple

import numpy as np
import torch

# stream ids: one per kind of random object, so adding draws to one object
# never changes another.
STREAM_BLOBS = 1
STREAM_NOISE = 2
STREAM_TF = 3
STREAM_CAMERAS = 4
STREAM_KD = 5
STREAM_TF_PERTURB = 6
STREAM_SELECT = 7
STREAM_GRAD = 8


def rng(seed: int, stream: int) -> np.random.Generator:
    """PCG64 generator for (base seed, stream id)."""
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([int(seed), int(stream)])))


# --------------------------------------------------------------------------
# volume geometry
# --------------------------------------------------------------------------

def default_spacing(dims: Sequence[int]) -> float:
    """World spacing so that the longest axis spans [0, 1]."""
    return 1.0 / (max(dims) - 1)


def world_extent(dims: Sequence[int], spacing: Optional[float] = None) -> np.ndarray:
    sp = default_spacing(dims) if spacing is None else spacing
    return np.array([(d - 1) * sp for d in dims], dtype=np.float64)


# --------------------------------------------------------------------------
# scalar fields
# --------------------------------------------------------------------------

@dataclass
class Blobs:
    centers: np.ndarray   # (n, 3) world coordinates
    sigmas: np.ndarray    # (n,)
    amps: np.ndarray      # (n,)


def blob_params(n: int, dims: Sequence[int], seed: int = 0,
                sigma_range=(0.05, 0.2), amp_range=(0.3, 1.0)) -> Blobs:
    """Gaussian blob parameters: centres uniform in the volume's box (the unit
    cube scaled to the world extent), widths and amplitudes uniform."""
    g = rng(seed, STREAM_BLOBS)
    ext = world_extent(dims)
    centers = g.uniform(0.0, 1.0, size=(n, 3)) * ext[None, :]
    sigmas = g.uniform(sigma_range[0], sigma_range[1], size=n)
    amps = g.uniform(amp_range[0], amp_range[1], size=n)
    return Blobs(centers, sigmas, amps)


def _axis_coords(n: int, sp: float, device) -> torch.Tensor:
    return torch.arange(n, device=device, dtype=torch.float64).to(torch.float32) * sp


def blob_field(dims: Sequence[int], blobs: Blobs, device="cpu", clamp=True, trunc: float = 6.0) -> torch.Tensor:
    """Sum of isotropic Gaussians, evaluated in float32, optionally clamped to
    [0, 1].  Blobs are truncated at `trunc` sigma (6: below 2e-8 of their
    amplitude)."""
    nx, ny, nz = dims
    sp = default_spacing(dims)
    out = torch.zeros((nz, ny, nx), dtype=torch.float32, device=device)
    xs = _axis_coords(nx, sp, device)
    ys = _axis_coords(ny, sp, device)
    zs = _axis_coords(nz, sp, device)
    for c, s, a in zip(blobs.centers, blobs.sigmas, blobs.amps):
        r = trunc * s
        lo = [max(0, int(math.floor((c[k] - r) / sp))) for k in range(3)]
        hi = [min(d, int(math.ceil((c[k] + r) / sp)) + 1) for k, d in enumerate(dims)]
        if any(h <= l for l, h in zip(lo, hi)):
            continue
        inv = float(1.0 / (2.0 * s * s))
        gx = torch.exp(-(xs[lo[0]:hi[0]] - float(c[0])) ** 2 * inv)
        gy = torch.exp(-(ys[lo[1]:hi[1]] - float(c[1])) ** 2 * inv)
        gz = torch.exp(-(zs[lo[2]:hi[2]] - float(c[2])) ** 2 * inv)
        out[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]] += float(a) * (
            gz[:, None, None] * gy[None, :, None] * gx[None, None, :])
    if clamp:
        out.clamp_(0.0, 1.0)
    return out


def _pcg_hash(v: torch.Tensor) -> torch.Tensor:
    """32-bit PCG output-permutation hash (RXS-M-XS) on int64 tensors holding
    unsigned 32-bit values (Jarzynski and Olano, "Hash Functions for GPU
    Rendering", JCGT 2020)."""
    m = 0xFFFFFFFF
    state = (v * 747796405 + 2891336453) & m
    word = (((state >> ((state >> 28) + 4)) ^ state) * 277803737) & m
    return ((word >> 22) ^ word) & m


def _lattice_value(ix, iy, iz, octave: int, seed: int) -> torch.Tensor:
    """Seeded lattice value in [0, 1) for integer lattice coordinates."""
    m = 0xFFFFFFFF
    h = _pcg_hash(torch.full_like(ix, (seed * 0x9E3779B1 + octave * 0x85EBCA77) & m))
    h = _pcg_hash((iz & m) ^ h)
    h = _pcg_hash((iy & m) ^ h)
    h = _pcg_hash((ix & m) ^ h)
    return h.to(torch.float64).to(torch.float32) * (1.0 / 4294967296.0)


def _smooth5(t: torch.Tensor) -> torch.Tensor:
    return t * t * t * (t * (t * 6.0 - 15.0) + 10.0)


def value_noise(dims: Sequence[int], octaves: int, seed: int = 0, f0: float = 4.0,
                device="cpu", normalize=True) -> torch.Tensor:
    """Multi-octave value noise: octave o has f0 * 2**o lattice cells per world
    unit and amplitude 0.5**o; lattice values come from a seeded PCG hash and
    are blended with a quintic smoothstep, separably (x, then y, then z).
    Normalised to [0, 1] by min/max."""
    nx, ny, nz = dims
    sp = default_spacing(dims)
    out = torch.zeros((nz, ny, nx), dtype=torch.float32, device=device)
    nseed = int(rng(seed, STREAM_NOISE).integers(0, 2 ** 31))
    coords = [_axis_coords(n, sp, device) for n in dims]
    for o in range(octaves):
        freq = f0 * (2 ** o)
        amp = 0.5 ** o
        idx, wts = [], []
        for c in coords:
            u = c * freq
            i = torch.floor(u)
            idx.append(i.to(torch.int64))
            wts.append(_smooth5(u - i))
        (ix, iy, iz), (wx, wy, wz) = idx, wts
        lat = [torch.arange(int(i.min()), int(i.max()) + 2, device=device, dtype=torch.int64) for i in idx]
        L = _lattice_value(lat[0][None, None, :], lat[1][None, :, None], lat[2][:, None, None], o, nseed)
        rx, ry, rz = ix - lat[0][0], iy - lat[1][0], iz - lat[2][0]
        T1 = L[:, :, rx] * (1.0 - wx) + L[:, :, rx + 1] * wx                      # (Lz, Ly, nx)
        T2 = T1[:, ry, :] * (1.0 - wy)[None, :, None] + T1[:, ry + 1, :] * wy[None, :, None]   # (Lz, ny, nx)
        del T1
        slab = max(1, (1 << 26) // (nx * ny))
        for z0 in range(0, nz, slab):
            z1 = min(nz, z0 + slab)
            out[z0:z1].add_(torch.lerp(T2[rz[z0:z1]], T2[rz[z0:z1] + 1], wz[z0:z1, None, None]), alpha=amp)
        del T2
    if normalize:
        out = _normalize01(out)
    return out


def _normalize01(f: torch.Tensor) -> torch.Tensor:
    lo = f.min()
    hi = f.max()
    return ((f - lo) / (hi - lo)).to(torch.float32)


def lognormal(f: torch.Tensor, k: float = 1.5) -> torch.Tensor:
    """Pointwise log-normal intermittency: exp(k * (n - mean(n))), renormalised
    to [0, 1]."""
    g = torch.exp(k * (f.to(torch.float32) - f.to(torch.float64).mean().to(torch.float32)))
    return _normalize01(g)


# named field recipes (dims are (nx, ny, nz)) ---------------------------------

def field_small(seed: int = 0, dims=(64, 64, 64), device="cpu") -> torch.Tensor:
    """Sum of 8 blobs, clamped to [0, 1]."""
    return blob_field(dims, blob_params(8, dims, seed), device=device, clamp=True)


def field_mid(seed: int = 0, dims=(512, 512, 512), device="cpu") -> torch.Tensor:
    """64 blobs plus 3-octave value noise (weight 0.5), min/max normalised."""
    b = blob_field(dims, blob_params(64, dims, seed), device=device, clamp=False)
    n = value_noise(dims, 3, seed, device=device)
    return _normalize01(b + 0.5 * n)


def field_turbulent(seed: int = 0, dims=(1024, 1024, 512), device="cpu") -> torch.Tensor:
    """5-octave value noise with log-normal amplitude."""
    return lognormal(value_noise(dims, 5, seed, device=device))


def field_diff(seed: int = 0, dims=(256, 256, 256), device="cpu") -> torch.Tensor:
    """16 blobs, clamped to [0, 1]."""
    return blob_field(dims, blob_params(16, dims, seed), device=device, clamp=True)


def field_large(seed: int = 0, dims=(2048, 2048, 2048), device="cpu") -> torch.Tensor:
    """4-octave value noise plus 256 small blobs (sigma U[0.01, 0.03],
    truncated at 5 sigma), min/max normalised."""
    b = blob_field(dims, blob_params(256, dims, seed, sigma_range=(0.01, 0.03)), device=device, clamp=False,
                   trunc=5.0)
    n = value_noise(dims, 4, seed, device=device)
    b.add_(n, alpha=0.5)
    del n
    return _normalize01_(b)


def _normalize01_(f: torch.Tensor) -> torch.Tensor:
    """In-place min/max normalisation (for fields too large to copy)."""
    lo = f.min()
    hi = f.max()
    return f.sub_(lo).div_(hi - lo)


# --------------------------------------------------------------------------
# transfer function
# --------------------------------------------------------------------------

def make_tf(seed: int = 1234, n: int = 256, n_ctrl: int = 8, transparent_below: float = 0.0) -> np.ndarray:
    """Piecewise-linear RGBA table of n entries at s_i = i / (n - 1).

    n_ctrl control points: sorted positions in [0, 1] with both endpoints
    pinned, RGB uniform in [0, 1], alpha uniform in [0, 1] times the position
    (an opacity ramp), linearly resampled to n entries.  With
    transparent_below > 0 the entries at s_i <= transparent_below get alpha
    exactly 0 (a classification that hides the low values).  Returns (n, 4)
    f32."""
    g = rng(seed, STREAM_TF)
    pos = np.sort(g.uniform(0.0, 1.0, size=n_ctrl - 2))
    pos = np.concatenate([[0.0], pos, [1.0]])
    rgb = g.uniform(0.0, 1.0, size=(n_ctrl, 3))
    a = g.uniform(0.0, 1.0, size=n_ctrl) * pos
    xs = np.arange(n, dtype=np.float64) / (n - 1)
    tab = np.empty((n, 4), dtype=np.float64)
    for ch in range(3):
        tab[:, ch] = np.interp(xs, pos, rgb[:, ch])
    tab[:, 3] = np.interp(xs, pos, a)
    if transparent_below > 0.0:
        tab[xs <= transparent_below, 3] = 0.0
    return tab.astype(np.float32)


def linear_tf(n: int = 256) -> np.ndarray:
    """RGBA table of n entries whose every channel is linear in s (no kink
    between the end entries): r = 0.2 + 0.6 s, g = 0.8 - 0.5 s,
    b = 0.3 + 0.4 s, alpha = 0.05 + 0.6 s.  Returns (n, 4) f32."""
    xs = np.arange(n, dtype=np.float64) / (n - 1)
    tab = np.stack([0.2 + 0.6 * xs, 0.8 - 0.5 * xs, 0.3 + 0.4 * xs, 0.05 + 0.6 * xs], -1)
    return tab.astype(np.float32)


def perturb_tf(tf: np.ndarray, seed: int = 0, sigma: float = 0.05) -> np.ndarray:
    """Target table for the differentiable workload: clamp(TF + N(0, sigma^2))."""
    g = rng(seed, STREAM_TF_PERTURB)
    return np.clip(tf + g.normal(0.0, sigma, size=tf.shape), 0.0, 1.0).astype(np.float32)


# --------------------------------------------------------------------------
# cameras
# --------------------------------------------------------------------------

@dataclass
class Camera:
    eye: Tuple[float, float, float]
    center: Tuple[float, float, float]
    up: Tuple[float, float, float]
    fovy_deg: float = 40.0

    def as_array(self) -> np.ndarray:
        return np.array([*self.eye, *self.center, *self.up, self.fovy_deg], dtype=np.float64)


def _up_for(direction: np.ndarray) -> Tuple[float, float, float]:
    d = direction / np.linalg.norm(direction)
    return (0.0, 1.0, 0.0) if abs(d[2]) > 0.99 else (0.0, 0.0, 1.0)


def camera_from_direction(dims: Sequence[int], direction, fovy_deg: float = 40.0,
                          distance_scale: float = 1.0) -> Camera:
    """Camera on the ray from the volume centre along `direction`, at the
    distance where the bounding sphere just fits the vertical field of view
    (radius / sin(fovy / 2)), looking at the centre."""
    ext = world_extent(dims)
    c = ext / 2.0
    r = float(np.linalg.norm(ext) / 2.0)
    d = np.asarray(direction, dtype=np.float64)
    d = d / np.linalg.norm(d)
    dist = distance_scale * r / math.sin(math.radians(fovy_deg) / 2.0)
    eye = c + dist * d
    return Camera(tuple(eye), tuple(c), _up_for(d), fovy_deg)


def orbit_cameras(dims: Sequence[int], n: int, seed: int = 0, fovy_deg: float = 40.0) -> List[Camera]:
    """n cameras on an orbit: azimuth 2 pi k / n plus one seeded phase,
    elevation uniform in [-30, 30] degrees."""
    g = rng(seed, STREAM_CAMERAS)
    phase = g.uniform(0.0, 2.0 * math.pi)
    cams = []
    for k in range(n):
        az = 2.0 * math.pi * k / n + phase
        el = math.radians(g.uniform(-30.0, 30.0))
        d = (math.cos(el) * math.cos(az), math.cos(el) * math.sin(az), math.sin(el))
        cams.append(camera_from_direction(dims, d, fovy_deg))
    return cams


def sphere_cameras(dims: Sequence[int], n: int, seed: int = 0, fovy_deg: float = 40.0) -> List[Camera]:
    """n view directions uniform on the unit sphere (normalised Gaussians)."""
    g = rng(seed, STREAM_CAMERAS)
    cams = []
    for _ in range(n):
        v = g.normal(size=3)
        cams.append(camera_from_direction(dims, v / np.linalg.norm(v), fovy_deg))
    return cams


def random_cameras(dims: Sequence[int], n: int, seed: int = 0, inside: bool = False,
                   fovy_deg: float = 40.0) -> List[Camera]:
    """Cameras for invariance tests: outside the volume at random directions
    and distances, or (inside=True) at random points inside the box looking at
    random targets."""
    g = rng(seed, STREAM_CAMERAS + 100)
    ext = world_extent(dims)
    cams = []
    for _ in range(n):
        if inside:
            eye = g.uniform(0.15, 0.85, size=3) * ext
            tgt = g.uniform(0.0, 1.0, size=3) * ext
            d = tgt - eye
            cams.append(Camera(tuple(eye), tuple(tgt), _up_for(d), fovy_deg))
        else:
            v = g.normal(size=3)
            cams.append(camera_from_direction(dims, v / np.linalg.norm(v), fovy_deg,
                                              distance_scale=g.uniform(0.8, 2.0)))
    return cams


# --------------------------------------------------------------------------
# partitions
# --------------------------------------------------------------------------

@dataclass
class Partition:
    """Half-open node ranges per rank plus the k-d tree that produced them.

    tree nodes: axis, split (node index), left, right; a child < 0 encodes
    leaf -(rank + 1)."""
    lo: np.ndarray            # (K, 3) int
    hi: np.ndarray            # (K, 3) int
    axis: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int32))
    split: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int32))
    left: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int32))
    right: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int32))

    @property
    def num_ranks(self) -> int:
        return int(self.lo.shape[0])


def regular_partition(dims: Sequence[int], splits: Sequence[int]) -> Partition:
    """splits[a] equal (as even as integer division allows) node ranges per
    axis; rank order is x fastest.  The tree splits x, then y, then z by
    halving the rank ranges recursively."""
    cuts = [[(k * dims[a]) // splits[a] for k in range(splits[a] + 1)] for a in range(3)]
    lo, hi = [], []
    for kz in range(splits[2]):
        for ky in range(splits[1]):
            for kx in range(splits[0]):
                lo.append([cuts[0][kx], cuts[1][ky], cuts[2][kz]])
                hi.append([cuts[0][kx + 1], cuts[1][ky + 1], cuts[2][kz + 1]])
    lo = np.array(lo, dtype=np.int32)
    hi = np.array(hi, dtype=np.int32)
    axis, split, left, right = [], [], [], []

    def rank_of(kx, ky, kz):
        return kx + splits[0] * (ky + splits[1] * kz)

    def build(r0, r1):  # r0/r1: per-axis brick index ranges [r0, r1)
        ext = [r1[a] - r0[a] for a in range(3)]
        if all(e == 1 for e in ext):
            return -(rank_of(r0[0], r0[1], r0[2]) + 1)
        a = max(range(3), key=lambda k: (ext[k] > 1, ext[k], -k))
        mid = r0[a] + ext[a] // 2
        node = len(axis)
        axis.append(a)
        split.append(cuts[a][mid])
        left.append(0)
        right.append(0)
        lr1 = list(r1)
        lr1[a] = mid
        rr0 = list(r0)
        rr0[a] = mid
        left[node] = build(r0, lr1)
        right[node] = build(rr0, r1)
        return node

    build([0, 0, 0], list(splits))
    return Partition(lo, hi, np.array(axis, np.int32), np.array(split, np.int32),
                     np.array(left, np.int32), np.array(right, np.int32))


def kd_partition(dims: Sequence[int], n_leaves: int, seed: int = 0,
                 frac=(0.3, 0.7)) -> Partition:
    """Repeatedly split the leaf with the most nodes (lowest rank on ties)
    along its longest axis (lowest axis on ties) at node index
    lo + round(u * (hi - lo)), u uniform in frac, until n_leaves leaves."""
    g = rng(seed, STREAM_KD)
    leaves = [(list([0, 0, 0]), list(dims))]
    # tree bookkeeping: leaf_node[rank] = (parent node, side) or None for root
    axis, split, left, right = [], [], [], []
    parent_of = [None]
    while len(leaves) < n_leaves:
        counts = [int(np.prod([h - l for l, h in zip(lo, hi)])) for lo, hi in leaves]
        r = int(np.argmax(counts))
        lo, hi = leaves[r]
        ext = [h - l for l, h in zip(lo, hi)]
        a = int(np.argmax(ext))
        if ext[a] < 2:
            raise ValueError("cannot split further")
        u = g.uniform(frac[0], frac[1])
        s = lo[a] + int(round(u * (hi[a] - lo[a])))
        s = min(max(s, lo[a] + 1), hi[a] - 1)
        node = len(axis)
        axis.append(a)
        split.append(s)
        new_rank = len(leaves)
        left.append(-(r + 1))
        right.append(-(new_rank + 1))
        if parent_of[r] is not None:
            p, side = parent_of[r]
            (left if side == 0 else right)[p] = node
        parent_of[r] = (node, 0)
        parent_of.append((node, 1))
        lhi = list(hi)
        lhi[a] = s
        rlo = list(lo)
        rlo[a] = s
        leaves[r] = (lo, lhi)
        leaves.append((rlo, hi))
    lo = np.array([l for l, _ in leaves], dtype=np.int32)
    hi = np.array([h for _, h in leaves], dtype=np.int32)
    if not axis:
        return Partition(lo, hi)
    return Partition(lo, hi, np.array(axis, np.int32), np.array(split, np.int32),
                     np.array(left, np.int32), np.array(right, np.int32))


def pixel_subsample(width: int, height: int, step: int = 4) -> np.ndarray:
    """Pixel indices y * width + x with x % step == 0 and y % step == 0."""
    ys, xs = np.meshgrid(np.arange(0, height, step), np.arange(0, width, step), indexing="ij")
    return (ys * width + xs).reshape(-1).astype(np.int32)
