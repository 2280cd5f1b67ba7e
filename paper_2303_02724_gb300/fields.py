"""Seeded synthetic scalar fields (inputs only; no extremum-graph arithmetic).

These generators stand in for the paper's Open SciVis volumes and Schwefel
samples (Sec. 6, Table 2, Table 3), which are not available here.  Both the
CUDA path and the CPU oracle are fed from this module; it imports nothing from
either of them.

All arrays are float32 (except those of ``typed_ties`` and ``quantise``, which
hold the requested element type), C-ordered with the LAST numpy axis fastest, which is
axis 0 of the grid (vertex index v = x0 + n0*(x1 + n1*(x2 + ...))).  So a 3D
field has numpy shape (n2, n1, n0) and ``extents`` = (n0, n1, n2).

Draw order is part of the recipe: for a sum of Gaussians, per Gaussian the
centre (one uniform per axis, axis 0 first), then the widths, then the
amplitude; after all Gaussians, the noise.  Gaussian sums are evaluated in
float64 (the Gaussians are axis-aligned, hence separable, so the sum is a
product of 1D tables contracted over the Gaussian index) and cast to float32.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field as dc_field

import numpy as np


@dataclass
class Field:
    values: np.ndarray            # float32, numpy shape = reversed(extents)
    extents: tuple                # axis 0 fastest
    name: str = ""
    meta: dict = dc_field(default_factory=dict)

    @property
    def d(self) -> int:
        return len(self.extents)

    @property
    def n(self) -> int:
        return int(np.prod(self.extents))


def _axis_tables(rng, extents, n_gauss, sigma_lo, sigma_hi, amp_lo, amp_hi,
                 isotropic):
    """Draw Gaussian parameters and return per-axis 1D tables (float64)."""
    d = len(extents)
    tables = [np.empty((n_gauss, extents[k]), np.float64) for k in range(d)]
    amps = np.empty(n_gauss, np.float64)
    for g in range(n_gauss):
        centre = [rng.uniform(0.0, extents[k]) for k in range(d)]
        if isotropic:
            s = rng.uniform(sigma_lo, sigma_hi)
            sig = [s] * d
        else:
            sig = [rng.uniform(sigma_lo, sigma_hi) for _ in range(d)]
        amps[g] = rng.uniform(amp_lo, amp_hi)
        for k in range(d):
            x = np.arange(extents[k], dtype=np.float64)
            tables[k][g] = np.exp(-0.5 * ((x - centre[k]) / sig[k]) ** 2)
    return tables, amps


def _contract(tables, amps, extents):
    """sum_g amps[g] * prod_k tables[k][g, x_k], numpy shape reversed(extents)."""
    d = len(extents)
    # acc[g, rest...] built from the fastest axis up; the slowest axis carries amps.
    acc = tables[0]                                    # (G, n0)
    for k in range(1, d - 1):
        acc = (tables[k][:, :, None] * acc[:, None, :]).reshape(acc.shape[0], -1)
    if d == 1:
        return (amps[:, None] * acc).sum(axis=0)
    slow = (tables[d - 1] * amps[:, None]).T           # (n_{d-1}, G)
    out = slow @ acc                                    # (n_{d-1}, prod of the rest)
    return out.reshape(tuple(reversed(extents)))


def gaussian_sum(extents, seed, n_gauss, sigma, amp, isotropic, noise,
                 rng=None, name=""):
    """Sum of axis-aligned Gaussians plus iid noise.

    sigma, amp: (lo, hi) uniform ranges.  noise: ("normal", std) or
    ("uniform", half_width) or None.
    """
    rng = np.random.default_rng(seed) if rng is None else rng
    extents = tuple(int(e) for e in extents)
    tables, amps = _axis_tables(rng, extents, n_gauss, sigma[0], sigma[1],
                                amp[0], amp[1], isotropic)
    f = _contract(tables, amps, extents)
    shape = tuple(reversed(extents))
    if noise is not None:
        kind, a = noise
        if kind == "normal":
            f = f + rng.normal(0.0, a, size=shape)
        elif kind == "uniform":
            f = f + rng.uniform(-a, a, size=shape)
        else:
            raise ValueError(kind)
    return Field(np.ascontiguousarray(f, dtype=np.float32).reshape(shape), extents, name,
                 {"seed": seed, "n_gauss": n_gauss})


def config_2d_256(seed=0, side=256):
    """2D side^2, 16 isotropic Gaussians (sigma U[4,16], amplitude U[0.5,1])
    plus iid normal noise of standard deviation 0.01."""
    return gaussian_sum((side, side), seed, 16, (4.0, 16.0), (0.5, 1.0), True,
                        ("normal", 0.01), name=f"2d_{side}x{side}_gauss16")


def config_3d_256(seed=1, side=256):
    """3D side^3, 64 anisotropic Gaussians (sigma U[6,30] per axis, amplitude
    U[0.3,1]) plus iid uniform noise in [-1e-3, 1e-3]."""
    return gaussian_sum((side, side, side), seed, 64, (6.0, 30.0), (0.3, 1.0), False,
                        ("uniform", 1e-3), name=f"3d_{side}^3_gauss64")


def grf(extents, seed, slope=-11.0 / 3.0, name=""):
    """Gaussian random field with isotropic power spectrum P(k) ~ k^slope.

    White N(0,1) noise (float32 draws) -> real FFT -> multiply by k^(slope/2),
    k = |integer wave vector|, the k = 0 mode set to 0 -> inverse FFT ->
    subtract the mean and divide by the standard deviation (both in float64)
    -> float32.
    """
    import scipy.fft as sfft
    extents = tuple(int(e) for e in extents)
    shape = tuple(reversed(extents))
    rng = np.random.default_rng(seed)
    w = rng.standard_normal(size=shape, dtype=np.float32)
    F = sfft.rfftn(w, workers=-1)
    del w
    k2 = None
    for ax, n in enumerate(shape):
        if ax == len(shape) - 1:
            kk = np.arange(n // 2 + 1, dtype=np.float32)
        else:
            kk = np.fft.fftfreq(n, d=1.0 / n).astype(np.float32)
        sh = [1] * len(shape)
        sh[ax] = kk.size
        term = (kk * kk).reshape(sh)
        k2 = term if k2 is None else k2 + term
    with np.errstate(divide="ignore"):
        amp = np.where(k2 > 0, k2 ** np.float32(slope / 4.0), np.float32(0.0)).astype(np.float32)
    F *= amp
    del amp, k2
    g = sfft.irfftn(F, s=shape, workers=-1)
    del F
    mean = float(np.mean(g, dtype=np.float64))
    std = float(np.std(g, dtype=np.float64))
    out = ((g.astype(np.float64) - mean) / std).astype(np.float32)
    return Field(np.ascontiguousarray(out), extents, name or f"grf_{'x'.join(map(str, extents))}",
                 {"seed": seed, "slope": slope})


def config_3d_512(seed=2, side=512):
    """3D side^3 Gaussian random field, P(k) ~ k^-11/3, zero mean, unit variance."""
    return grf((side, side, side), seed, -11.0 / 3.0, name=f"3d_{side}^3_grf")


def _loguniform_side(rng, lo, hi):
    return int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))


def batch_specs(seed=3, count=256, scale=1.0):
    """Shapes of the uneven batch: per field, d = 2 or 3 with probability 1/2,
    side log-uniform in 64..2048 (2D) or 32..256 (3D), U{4..64} Gaussians, and
    a seed for its values.  ``scale`` < 1 shrinks every side (quick tests)
    without changing any draw."""
    rng = np.random.default_rng(seed)
    specs = []
    for _ in range(count):
        d = 2 if rng.uniform() < 0.5 else 3
        side = _loguniform_side(rng, 64, 2048) if d == 2 else _loguniform_side(rng, 32, 256)
        side = max(2, int(round(side * scale)))
        ng = int(rng.integers(4, 65))
        fseed = int(rng.integers(0, 2 ** 63 - 1))
        specs.append(((side,) * d, fseed, ng))
    return specs


def batch_field(extents, fseed, n_gauss, name=""):
    """One batch member: 2D isotropic sigma U[4,16], amplitude U[0.5,1]; 3D
    sigma U[6,30] per axis, amplitude U[0.3,1]; plus uniform noise in
    [-1e-3, 1e-3]."""
    if len(extents) == 2:
        return gaussian_sum(extents, fseed, n_gauss, (4.0, 16.0), (0.5, 1.0), True,
                            ("uniform", 1e-3), name=name)
    return gaussian_sum(extents, fseed, n_gauss, (6.0, 30.0), (0.3, 1.0), False,
                        ("uniform", 1e-3), name=name)


def batch_fields(seed=3, count=256, scale=1.0):
    """The uneven batch of ``batch_specs`` with its values."""
    return [batch_field(e, s, g, name=f"b{i}_{len(e)}d_{e[0]}")
            for i, (e, s, g) in enumerate(batch_specs(seed, count, scale))]


SERVE_SIGMA = {2: (4.0, 16.0), 3: (6.0, 30.0), 4: (2.0, 8.0)}
SERVE_AMP = {2: (0.5, 1.0), 3: (0.3, 1.0), 4: (0.3, 1.0)}


def serve_requests(seed=4, count=4096, n_lo=1e4, n_hi=1e7):
    """Request shapes for the served stream: d uniform in {2,3,4}, vertex count
    log-uniform in [n_lo, n_hi], side = round(N^(1/d)), U{4..64} Gaussians.
    Returns a list of (extents, field_seed, n_gauss); values come from
    ``serve_field``."""
    rng = np.random.default_rng(seed)
    reqs = []
    for i in range(count):
        d = int(rng.integers(2, 5))
        n = math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))
        side = max(2, int(round(n ** (1.0 / d))))
        ng = int(rng.integers(4, 65))
        fseed = int(rng.integers(0, 2 ** 63 - 1))
        reqs.append(((side,) * d, fseed, ng))
    return reqs


def serve_field(extents, fseed, n_gauss):
    d = len(extents)
    return gaussian_sum(extents, fseed, n_gauss, SERVE_SIGMA[d], SERVE_AMP[d], d != 2,
                        ("uniform", 1e-3), name=f"req_{d}d_{extents[0]}")


def white_noise(extents, seed, dist="normal"):
    """iid field (tie-free almost surely) for density and symmetry checks."""
    rng = np.random.default_rng(seed)
    shape = tuple(reversed(tuple(extents)))
    if dist == "normal":
        v = rng.standard_normal(size=shape)
    else:
        v = rng.uniform(size=shape)
    return Field(np.ascontiguousarray(v, dtype=np.float32), tuple(extents), f"white_{dist}")


def integer_ties(extents, seed, levels=4):
    """Small-integer field with heavy ties, to exercise the index tie-break."""
    rng = np.random.default_rng(seed)
    shape = tuple(reversed(tuple(extents)))
    v = rng.integers(0, levels, size=shape).astype(np.float32)
    return Field(np.ascontiguousarray(v), tuple(extents), f"ties{levels}")


def schwefel(extents, seed=5, lo=-500.0, hi=500.0):
    """Schwefel function sum_i -x_i sin(sqrt|x_i|) sampled on a regular grid over
    [lo, hi]^d (the domain is not stated for the paper's Table 3; this one is the
    function's usual search domain).  The seed only shifts the sampling window
    by a fraction of a cell."""
    rng = np.random.default_rng(seed)
    extents = tuple(int(e) for e in extents)
    d = len(extents)
    axes = []
    for k in range(d):
        h = (hi - lo) / max(1, extents[k] - 1)
        x = lo + h * (np.arange(extents[k], dtype=np.float64) + rng.uniform(-0.25, 0.25))
        axes.append(-x * np.sin(np.sqrt(np.abs(x))))
    acc = np.zeros(tuple(reversed(extents)), np.float64)
    for k in range(d):
        sh = [1] * d
        sh[d - 1 - k] = extents[k]
        acc = acc + axes[k].reshape(sh)
    return Field(np.ascontiguousarray(acc, dtype=np.float32), extents, f"schwefel{d}d")


# Element types a field may have (Sec. 5 lists 8- to 64-bit integers and
# floats).  Per type, values on both sides of every boundary a wrong
# comparison would trip over: the extremes, both sides of the sign bit, and
# neighbours that float32 (or float64) cannot tell apart.
ELEMENT_TYPES = ("float32", "float64", "int8", "uint8", "int16", "uint16", "int32", "uint32",
                 "int64", "uint64")
EDGE_VALUES = {
    "float32": [-math.inf, -3.0e38, -1.0, -0.0, 0.0, 1.0e-45, 1.0, 1.0 + 2.0 ** -23, 3.0e38, math.inf],
    "float64": [-math.inf, -1.0e300, -1.0, -0.0, 0.0, 5.0e-324, 1.0, 1.0 + 2.0 ** -52, 1.0 + 2.0 ** -30,
                1.0e300, math.inf],
    "int8": [-128, -127, -1, 0, 1, 126, 127],
    "uint8": [0, 1, 127, 128, 129, 254, 255],
    "int16": [-32768, -32767, -1, 0, 1, 32766, 32767],
    "uint16": [0, 1, 32767, 32768, 65534, 65535],
    "int32": [-2 ** 31, -2 ** 31 + 1, -1, 0, 1, 2 ** 24, 2 ** 24 + 1, 2 ** 31 - 1],
    "uint32": [0, 1, 2 ** 24, 2 ** 24 + 1, 2 ** 31 - 1, 2 ** 31, 2 ** 32 - 2, 2 ** 32 - 1],
    "int64": [-2 ** 63, -2 ** 63 + 1, -1, 0, 1, 2 ** 53, 2 ** 53 + 1, 2 ** 63 - 1],
    "uint64": [0, 1, 2 ** 53, 2 ** 53 + 1, 2 ** 63 - 1, 2 ** 63, 2 ** 64 - 2, 2 ** 64 - 1],
}


def typed_ties(extents, seed, dtype):
    """Field of element type ``dtype`` drawn uniformly from that type's
    EDGE_VALUES: heavy ties plus values that only an exact comparison in the
    type itself orders correctly."""
    dt = np.dtype(dtype)
    rng = np.random.default_rng(seed)
    shape = tuple(reversed(tuple(extents)))
    table = np.array(EDGE_VALUES[dt.name], dtype=dt)
    v = table[rng.integers(0, table.size, size=shape)]
    return Field(np.ascontiguousarray(v), tuple(extents), f"edges_{dt.name}")


def quantise(field: Field, dtype, levels=None) -> Field:
    """The same field in element type ``dtype``: integers get the values
    rescaled affinely onto [lo, lo + levels - 1] (default: the type's whole
    range, capped at 2^52 levels so that the float64 arithmetic stays exact)
    and rounded, so narrow types form plateaus; float64 gets the float32
    values widened (every float32 is a float64)."""
    dt = np.dtype(dtype)
    v = np.asarray(field.values, np.float64)
    if dt.kind == "f":
        out = v.astype(dt)
    else:
        info = np.iinfo(dt)
        n = min(int(info.max) - int(info.min) + 1, 2 ** 52) if levels is None else int(levels)
        lo, hi = float(v.min()), float(v.max())
        q = np.rint((v - lo) / (hi - lo if hi > lo else 1.0) * (n - 1))
        if info.min < 0:
            out = (q.astype(np.int64) + (-(n // 2))).astype(dt)  # centred on zero
        else:
            out = q.astype(np.uint64).astype(dt)
    return Field(np.ascontiguousarray(out), field.extents, f"{field.name}_{dt.name}", dict(field.meta))
