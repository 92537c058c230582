"""Seeded synthetic scalar fields shaped like the paper's workloads.

The paper evaluates on CESM climate fields (Section V-A, Table I), which are not
available here.  These generators build stand-ins with the shapes, value
distributions and smoothness of those workloads (2D climate-like Gaussian random
fields, a 3D turbulence-like log-normal field, a sum of anisotropic Gaussian
bumps) plus the mixed batches and request streams of the batched and served
forms.

This module holds no part of the compression method: it only makes inputs, so
that the oracle and the CUDA path can be fed identical bytes.  Every generator
is a pure function of its arguments (shape, spectral slope, seed); fields are
float32, row-major with x (``dims[0]``) fastest, returned as a torch tensor of
shape ``(nz, ny, nx)`` or ``(ny, nx)``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import torch


def _generator(seed: int, device) -> torch.Generator:
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    return g


def gaussian_bumps_2d(ny: int = 256, nx: int = 256, count: int = 40,
                      seed: int = 1, noise: float = 1e-3) -> torch.Tensor:
    """Sum of ``count`` rotated anisotropic Gaussians plus uniform noise.

    Centres uniform over the grid, amplitudes U[-1, 1], widths U[4, 32] pixels
    per principal axis, rotation U[0, pi); noise U[-noise, +noise].  Built in
    float64 with numpy (small sizes only), returned as float32 on the CPU.
    """
    rng = np.random.default_rng(seed)
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    f = np.zeros((ny, nx), np.float64)
    for _ in range(count):
        cx, cy = rng.uniform(0, nx), rng.uniform(0, ny)
        amp = rng.uniform(-1.0, 1.0)
        sx, sy = rng.uniform(4.0, 32.0), rng.uniform(4.0, 32.0)
        th = rng.uniform(0.0, math.pi)
        c, s = math.cos(th), math.sin(th)
        u = (x - cx) * c + (y - cy) * s
        v = -(x - cx) * s + (y - cy) * c
        f += amp * np.exp(-(u * u / (2 * sx * sx) + v * v / (2 * sy * sy)))
    f += rng.uniform(-noise, noise, size=f.shape)
    return torch.from_numpy(f.astype(np.float32))


def grf(shape, psd_slope: float, seed: int, device="cpu",
        dtype=torch.float32) -> torch.Tensor:
    """Periodic Gaussian random field with isotropic power spectral density
    P(k) proportional to k**psd_slope (k in cycles per box), zero mean, unit variance.

    White Gaussian noise is drawn with a seeded torch generator on ``device``,
    filtered by sqrt(P(k)) in Fourier space and transformed back.  The field is
    periodic along every axis of ``shape``.
    """
    shape = tuple(int(s) for s in shape)
    g = _generator(seed, device)
    white = torch.randn(shape, generator=g, device=device, dtype=dtype)
    spec = torch.fft.rfftn(white)
    del white
    ks = []
    for ax, n in enumerate(shape):
        if ax == len(shape) - 1:
            k = torch.fft.rfftfreq(n, d=1.0 / n, device=device)
        else:
            k = torch.fft.fftfreq(n, d=1.0 / n, device=device)
        view = [1] * len(shape)
        view[ax] = -1
        ks.append(k.to(dtype).reshape(view))
    k2 = ks[0] ** 2
    for k in ks[1:]:
        k2 = k2 + k ** 2
    k2[(0,) * len(shape)] = 1.0
    amp = k2 ** (psd_slope / 4.0)          # sqrt(k^slope) = (k^2)^(slope/4)
    amp[(0,) * len(shape)] = 0.0
    spec = spec * amp
    del amp, k2
    f = torch.fft.irfftn(spec, s=shape)
    del spec
    f = f - f.mean()
    f = f / f.std()
    return f.to(torch.float32).contiguous()


def climate_2d(ny: int = 1800, nx: int = 3600, seed: int = 2, device="cpu",
               psd_slope: float = -3.0) -> torch.Tensor:
    """Climate-like 2D field: a GRF with 2D power spectrum k^-3 generated on an
    nx-by-nx periodic box and cropped to ny rows, so it is periodic in x only
    (like a latitude-longitude grid)."""
    big = grf((max(nx, ny), nx), psd_slope, seed, device)
    return big[:ny].contiguous()


def turbulence_3d(n: int = 512, seed: int = 3, device="cpu",
                  energy_slope: float = -5.0 / 3.0) -> torch.Tensor:
    """Turbulence-like 3D density: a GRF whose shell-summed (energy) spectrum
    follows k^energy_slope (Kolmogorov -5/3, i.e. a 3D power spectral density
    k^(energy_slope-2)), standardised and exponentiated so the values are
    positive and right-skewed like a density field."""
    g = grf((n, n, n), energy_slope - 2.0, seed, device)
    return torch.exp(g)


def mixed_field(ndim: int, side: int, energy_slope: float, seed: int,
                device="cpu") -> torch.Tensor:
    """One member of a mixed batch: a GRF of the given dimensionality whose
    shell-summed spectrum follows k^energy_slope (2D: PSD k^(s-1); 3D: k^(s-2))."""
    shape = (side,) * ndim
    return grf(shape, energy_slope - (ndim - 1), seed, device)


# ---------------------------------------------------------------- workloads

@dataclass(frozen=True)
class FieldSpec:
    """One synthetic field: how to build it and which error bound to use."""
    name: str
    ndim: int
    dims: tuple          # (nx, ny[, nz]) -- x fastest
    kind: str            # "bumps" | "climate" | "turb" | "mixed"
    seed: int
    eb_mode: str         # "abs_range" (eb * (max-min) given as ABS) | "rel"
    eb: float
    slope: float = 0.0

    @property
    def n(self) -> int:
        return int(np.prod(self.dims))

    @property
    def nbytes(self) -> int:
        return 4 * self.n

    def shape(self):
        return tuple(reversed(self.dims))

    def make(self, device="cpu") -> torch.Tensor:
        if self.kind == "bumps":
            return gaussian_bumps_2d(self.dims[1], self.dims[0], seed=self.seed).to(device)
        if self.kind == "climate":
            return climate_2d(self.dims[1], self.dims[0], seed=self.seed, device=device)
        if self.kind == "turb":
            assert self.dims[0] == self.dims[1] == self.dims[2]
            return turbulence_3d(self.dims[0], seed=self.seed, device=device)
        if self.kind == "mixed":
            return mixed_field(self.ndim, self.dims[0], self.slope, self.seed, device)
        raise ValueError(self.kind)


def bumps_256(seed: int = 1) -> FieldSpec:
    """256x256 sum of 40 Gaussian bumps; absolute bound 1e-3 of the value range."""
    return FieldSpec("bumps256", 2, (256, 256), "bumps", seed, "abs_range", 1e-3)


def climate_1800x3600(eb: float, seed: int = 2) -> FieldSpec:
    return FieldSpec(f"climate1800x3600_rel{eb:g}", 2, (3600, 1800), "climate", seed, "rel", eb)


def turb_512(eb: float, seed: int = 3, n: int = 512) -> FieldSpec:
    return FieldSpec(f"turb{n}^3_rel{eb:g}", 3, (n, n, n), "turb", seed, "rel", eb)


def mixed_batch(count: int = 96, seed: int = 1000, side2=(128, 4096), side3=(64, 384),
                ebs=(1e-2, 1e-3, 1e-4)):
    """``count`` fields, half 2D and half 3D, sides log-uniform over the given
    ranges, energy slope U[-3, -5/3], relative bound drawn from ``ebs``."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        ndim = 2 if i % 2 == 0 else 3
        lo, hi = side2 if ndim == 2 else side3
        side = int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
        slope = float(rng.uniform(-3.0, -5.0 / 3.0))
        eb = float(ebs[int(rng.integers(len(ebs)))])
        out.append(FieldSpec(f"mixed{i}", ndim, (side,) * ndim, "mixed", seed + i, "rel", eb, slope))
    return out


@dataclass(frozen=True)
class Request:
    """One served request: arrival time (s), operation, field and bound."""
    rid: int
    t_arrive: float
    op: str              # "compress" | "decompress"
    spec: FieldSpec


def request_stream(count: int = 2000, rate_hz: float = 100.0, seed: int = 7,
                   min_bytes: int = 64 << 10, max_bytes: int = 1 << 30):
    """Poisson arrivals at ``rate_hz``; field size log-uniform in bytes between
    ``min_bytes`` and ``max_bytes`` (2D side sqrt(bytes/4), 3D side cbrt(bytes/4)),
    2D/3D 50/50, relative bound log-uniform in [1e-5, 1e-2], compress/decompress
    50/50, per-request seeds."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(count):
        t += float(rng.exponential(1.0 / rate_hz))
        nbytes = math.exp(rng.uniform(math.log(min_bytes), math.log(max_bytes)))
        ndim = 2 if rng.uniform() < 0.5 else 3
        side = max(4, int(round((nbytes / 4.0) ** (1.0 / ndim))))
        eb = float(10 ** rng.uniform(-5, -2))
        op = "compress" if rng.uniform() < 0.5 else "decompress"
        slope = -3.0 if i % 2 == 0 else -5.0 / 3.0
        spec = FieldSpec(f"req{i}", ndim, (side,) * ndim, "mixed", 5000 + i, "rel", eb, slope)
        out.append(Request(i, t, op, spec))
    return out


def adversarial_small(seed: int, dims) -> torch.Tensor:
    """Small fields full of ties and near-ties: integers from a narrow alphabet
    scaled by a small step, so that many neighbours share values or bins."""
    rng = np.random.default_rng(seed)
    shape = tuple(reversed(dims))
    a = rng.integers(-3, 4, size=shape).astype(np.float32) * np.float32(0.37)
    a += rng.choice(np.array([0.0, 1e-7, -1e-7, 2.5e-3], np.float32), size=shape)
    return torch.from_numpy(a.astype(np.float32))
