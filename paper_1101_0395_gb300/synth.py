"""Seeded synthetic RGB8 images that stand in for natural test images.

This module only makes inputs. It holds none of the quantizer's arithmetic and
is the one module that both the CUDA path's tests and the FP64 oracle's tests
draw their images from.

Recipe (a piecewise-smooth image with sensor-like noise):

* ``R`` region sites are drawn uniformly over the image; every pixel belongs to
  the region of its nearest site (a Voronoi partition).
* Each region has a uniform-random RGB mean and a smooth colour field: a random
  linear ramp plus one low-frequency sinusoid per channel, of overall scale
  ``sigma_b * field_gain`` (0-255 units) across a region.  The gain (1/6) was
  calibrated so that the unique-colour fraction lands in the 25-60 % range of
  natural photographs (a full-scale field plus per-pixel noise makes almost
  every pixel unique).
* Optional global ramps (``global_ramp`` units from edge to edge) cross all
  regions, as in large photographs with lighting gradients.
* Every pixel gets Gaussian noise of standard deviation ``sigma_n``.  Camera noise
  in 8-bit images is mostly shared by the three channels (demosaicing mixes
  them), so the draw is ``sigma_n * (sqrt(rho) * n_lum + sqrt(1 - rho) * n_c)``
  with luminance correlation ``rho``.
* Values are rounded half-to-even and clamped to 0..255.

All randomness comes from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014): the n-th output of the generator
seeded with ``seed`` is ``mix64(seed + n * 0x9E3779B97F4A7C15)``.  Independent
streams use ``n = stream * 2**32 + i + 1``.  Normal deviates use the Box-Muller
transform in FP64.  The same seed gives the same image on any machine.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Dict, List, Tuple

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix64(z: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def splitmix_stream(seed: int, stream: int, count: int, start: int = 0) -> np.ndarray:
    """Outputs ``start .. start+count-1`` of stream ``stream`` as uint64."""
    n = (np.uint64(stream) << np.uint64(32)) + np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + n * _GAMMA
    return _mix64(z)


def uniform(seed: int, stream: int, count: int) -> np.ndarray:
    """FP64 uniforms in [0, 1) from the top 53 bits."""
    return (splitmix_stream(seed, stream, count) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normal(seed: int, stream: int, count: int) -> np.ndarray:
    """Standard normals by Box-Muller (one deviate per uniform pair)."""
    u = uniform(seed, stream, 2 * count)
    u1 = 1.0 - u[0::2]  # (0, 1]
    u2 = u[1::2]
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)


def _nearest_site(xs: np.ndarray, ys: np.ndarray, sx: np.ndarray, sy: np.ndarray) -> np.ndarray:
    """Index of the nearest site per pixel (lowest index on exact ties)."""
    try:
        from scipy.spatial import cKDTree  # type: ignore

        tree = cKDTree(np.stack([sx, sy], axis=1))
        _, idx = tree.query(np.stack([xs, ys], axis=1), k=1)
        return idx.astype(np.int32)
    except ImportError:  # pragma: no cover - scipy is present on both machines
        out = np.empty(xs.shape[0], dtype=np.int32)
        step = max(1, (1 << 22) // max(1, sx.shape[0]))
        for a in range(0, xs.shape[0], step):
            d = (xs[a:a + step, None] - sx[None, :]) ** 2 + (ys[a:a + step, None] - sy[None, :]) ** 2
            out[a:a + step] = np.argmin(d, axis=1)
        return out


FIELD_GAIN = 1.0 / 6.0
NOISE_RHO = 0.99


def image(height: int, width: int, regions: int, sigma_b: float, sigma_n: float, seed: int,
          global_ramp: float = 0.0, rho: float = NOISE_RHO, field_gain: float = FIELD_GAIN) -> np.ndarray:
    """One packed HWC uint8 image of shape (height, width, 3)."""
    h, w, r = int(height), int(width), int(regions)
    s = seed
    site = uniform(s, 1, 2 * r)
    sx, sy = site[0::2] * w, site[1::2] * h
    mean = uniform(s, 2, 3 * r).reshape(r, 3) * 255.0
    g = normal(s, 3, 6 * r).reshape(r, 3, 2) * 0.5          # ramp slopes per channel
    amp = normal(s, 4, 3 * r).reshape(r, 3) * 0.9            # sinusoid amplitude per channel
    phase = uniform(s, 5, 3 * r).reshape(r, 3) * (2.0 * math.pi)
    fq = 0.5 + uniform(s, 6, r) * 1.5                        # cycles per region diameter
    th = uniform(s, 7, r) * (2.0 * math.pi)
    gr = normal(s, 8, 6).reshape(3, 2) * global_ramp
    scale = math.sqrt(h * w / r)                             # typical region diameter (px)

    out = np.empty((h, w, 3), dtype=np.uint8)
    rows_per = max(1, (1 << 20) // w)
    n_lum_all = normal(s, 10, h * w)
    n_ch_all = normal(s, 11, 3 * h * w).reshape(h * w, 3)
    for y0 in range(0, h, rows_per):
        y1 = min(h, y0 + rows_per)
        yy, xx = np.meshgrid(np.arange(y0, y1, dtype=np.float64) + 0.5,
                             np.arange(w, dtype=np.float64) + 0.5, indexing="ij")
        xs, ys = xx.ravel(), yy.ravel()
        lab = _nearest_site(xs, ys, sx, sy)
        u = (xs - sx[lab]) / scale
        v = (ys - sy[lab]) / scale
        arg = 2.0 * math.pi * fq[lab] * (u * np.cos(th[lab]) + v * np.sin(th[lab]))
        a, b = y0 * w, y1 * w
        lum = n_lum_all[a:b]
        val = np.empty((xs.shape[0], 3), dtype=np.float64)
        for c in range(3):
            fld = g[lab, c, 0] * u + g[lab, c, 1] * v
            fld += amp[lab, c] * math.sqrt(2.0) * np.sin(arg + phase[lab, c])
            v_c = mean[lab, c] + (sigma_b * field_gain) * fld
            if global_ramp:
                v_c += gr[c, 0] * (xs / w - 0.5) + gr[c, 1] * (ys / h - 0.5)
            v_c += sigma_n * (math.sqrt(rho) * lum + math.sqrt(1.0 - rho) * n_ch_all[a:b, c])
            val[:, c] = v_c
        out[y0:y1] = np.clip(np.rint(val), 0, 255).astype(np.uint8).reshape(y1 - y0, w, 3)
    return out


def unique_count(img: np.ndarray) -> int:
    """Number of distinct 24-bit colours (input bookkeeping only)."""
    p = img.reshape(-1, 3).astype(np.uint32)
    key = (p[:, 0] << 16) | (p[:, 1] << 8) | p[:, 2]
    return int(np.unique(key).shape[0])


@dataclass(frozen=True)
class Workload:
    """A named synthetic workload: image recipe plus quantizer settings."""
    name: str
    height: int
    width: int
    regions: int
    sigma_b: float
    sigma_n: float
    global_ramp: float
    ks: Tuple[int, ...]
    eps: float = 1e-4
    max_iter: int = 100
    unique_range: Tuple[int, int] = (0, 1 << 24)

    def make(self, index: int = 0) -> np.ndarray:
        return image(self.height, self.width, self.regions, self.sigma_b, self.sigma_n,
                     seed_for(self.name, index), self.global_ramp)


_CONFIG_INDEX = {"plain_256": 0, "paper_512": 1, "large_4096": 2, "batched": 3, "serving": 4}


def seed_for(name: str, index: int = 0) -> int:
    """Image seed: 1101 + workload index + image index."""
    return 1101 + _CONFIG_INDEX[name] * 100003 + index


WORKLOADS: Dict[str, Workload] = {
    # one 256x256 image, 48 regions, colour scale 12, noise 4, K = 16
    "plain_256": Workload("plain_256", 256, 256, 48, 12.0, 4.0, 0.0, (16,),
                          unique_range=(8_000, 40_000)),
    # 512x512 images, 96 regions, colour scale 12, noise 6, K in {32, 64, 128, 256}
    "paper_512": Workload("paper_512", 512, 512, 96, 12.0, 6.0, 0.0, (32, 64, 128, 256),
                          unique_range=(60_000, 150_000)),
    # 4096x4096 (16.7 Mpx), 512 regions plus global ramps, K = 256
    "large_4096": Workload("large_4096", 4096, 4096, 512, 12.0, 6.0, 60.0, (256,),
                           unique_range=(1_000_000, 4_000_000)),
}


@dataclass
class BatchSpec:
    """Uneven batch: side log-uniform in [lo, hi], aspect in [0.5, 2], K from ``ks``."""
    sizes: List[Tuple[int, int]] = field(default_factory=list)
    ks: List[int] = field(default_factory=list)
    seeds: List[int] = field(default_factory=list)


def batch_spec(count: int, side_lo: int = 64, side_hi: int = 2048,
               ks: Tuple[int, ...] = (16, 32, 64, 128, 256), seed: int = 3101,
               k_uniform_range: Tuple[int, int] | None = None) -> BatchSpec:
    """Image shapes and palette sizes for a batch of ``count`` uneven images."""
    u = uniform(seed, 20, 3 * count).reshape(count, 3)
    spec = BatchSpec()
    for i in range(count):
        side = math.exp(math.log(side_lo) + u[i, 0] * (math.log(side_hi) - math.log(side_lo)))
        aspect = math.exp(math.log(0.5) + u[i, 1] * (math.log(2.0) - math.log(0.5)))
        hh = max(8, int(round(side / math.sqrt(aspect))))
        ww = max(8, int(round(side * math.sqrt(aspect))))
        if k_uniform_range is not None:
            lo, hi = k_uniform_range
            k = lo + min(hi - lo, int(u[i, 2] * (hi - lo + 1)))
        else:
            k = ks[min(len(ks) - 1, int(u[i, 2] * len(ks)))]
        spec.sizes.append((hh, ww))
        spec.ks.append(k)
        spec.seeds.append(seed * 7919 + i)
    return spec


def batch_image(h: int, w: int, seed: int) -> np.ndarray:
    """One batch member: the 512x512 recipe scaled with area (regions ~ area)."""
    regions = max(4, int(round(96 * (h * w) / (512 * 512))))
    return image(h, w, regions, 12.0, 6.0, seed)
