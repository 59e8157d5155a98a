"""Seeded synthetic HI cubes: the inputs both the CUDA path and the oracle read.

This module only draws inputs.  It holds none of the source finder's own
arithmetic (no filter taps, no convolution of the method, no statistics): the
beam that correlates the noise is applied as a product in Fourier space, and
sources are analytic Gaussian blobs added to the cube.

The paper measured on a simulated survey cube that is not available here
(Sec. 4: 2048 x 2048 x 4096 voxels, concatenated four times along frequency).
These workloads stand in for it, scaled to one GPU.  Layout is cube[x][y][z]
with z (frequency) contiguous (Sec. 3.1).

Recipe (per workload below):
  noise  i.i.d. N(0, 1) from a seeded torch generator on the requested device;
         optionally correlated per channel by a circular 2D Gaussian beam
         (transfer function exp(-2 pi^2 sigma^2 |f|^2) on the x-y FFT) and
         rescaled to unit standard deviation by the exact discrete factor
         sqrt(mean |H|^2); optionally scaled per channel by a noise sigma rising
         linearly along z;
  sources  n blobs A exp(-(dx^2+dy^2)/(2 ss^2) - dz^2/(2 sf^2)) with centres
         uniform over the cube, ss ~ U[1,3] px, sf ~ U[2,10] channels,
         A = U[peak_lo, peak_hi] * noise sigma at the centre channel, added on
         the box of +-5 sigma around the centre (clipped to the cube);
         parameters from numpy PCG64(seed + 1).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import torch


@dataclass(frozen=True)
class Workload:
    """One synthetic workload: cube recipe plus the detection settings."""
    name: str
    shape: tuple[int, int, int]
    seed: int
    n_sources: int
    peak: tuple[float, float]
    beam_sigma: float | None
    noise_sigma: tuple[float, float] = (1.0, 1.0)
    bank: tuple[tuple[float, float], ...] = ((1.0, 2.0),)
    truncation: float = 3.0
    window: tuple[int, int, int] = (16, 16, 32)
    k: float = 4.0
    extra: dict = field(default_factory=dict)

    @property
    def voxels(self) -> int:
        return int(self.shape[0]) * int(self.shape[1]) * int(self.shape[2])


BANK6 = ((0.0, 2.0), (0.0, 6.0), (1.5, 2.0), (1.5, 6.0), (3.0, 2.0), (3.0, 6.0))

# Plain method, tiny: the oracle finishes it in seconds.
TINY = Workload("tiny-64x64x128-1filter", (64, 64, 128), 0, 8, (0.5, 3.0), None,
                bank=((1.0, 2.0),), window=(16, 16, 32))
# Survey tile, FP32, 6-filter bank: the throughput workload.
TILE = Workload("tile-512x512x1024-6filters", (512, 512, 1024), 1, 200, (0.3, 5.0), 1.5,
                bank=BANK6, window=(32, 32, 64))
# Precision workload: larger cube, noise sigma rising 0.8 -> 1.5 along z.
PRECISION = Workload("precision-1024x1024x2048-6filters", (1024, 1024, 2048), 2, 1000,
                     (0.3, 5.0), 1.5, noise_sigma=(0.8, 1.5), bank=BANK6, window=(32, 32, 64))

WORKLOADS = {w.name: w for w in (TINY, TILE, PRECISION)}


def _beam(noise: torch.Tensor, sigma: float) -> torch.Tensor:
    """Correlate each channel by a circular Gaussian beam, keep unit variance."""
    nx, ny, _ = noise.shape
    dev = noise.device
    fx = torch.fft.fftfreq(nx, device=dev, dtype=torch.float64)
    fy = torch.fft.rfftfreq(ny, device=dev, dtype=torch.float64)
    fy_full = torch.fft.fftfreq(ny, device=dev, dtype=torch.float64)
    c = -2.0 * math.pi ** 2 * sigma ** 2
    h = torch.exp(c * (fx[:, None] ** 2 + fy[None, :] ** 2))
    h_full = torch.exp(c * (fx[:, None] ** 2 + fy_full[None, :] ** 2))
    scale = 1.0 / math.sqrt(float((h_full ** 2).mean()))
    spec = torch.fft.rfft2(noise, dim=(0, 1))
    spec *= (h * scale).to(torch.complex64)[:, :, None]
    return torch.fft.irfft2(spec, s=(nx, ny), dim=(0, 1)).to(torch.float32)


def _noise_sigma_at(z: np.ndarray | float, nz: int, lohi: tuple[float, float]):
    lo, hi = lohi
    if nz <= 1:
        return lo
    return lo + (hi - lo) * np.asarray(z, dtype=np.float64) / (nz - 1)


def make_cube(shape, seed: int, n_sources: int, peak=(0.5, 3.0), beam_sigma=None,
              noise_sigma=(1.0, 1.0), device="cpu") -> torch.Tensor:
    """Seeded float32 cube [x][y][z] on `device` following the module recipe."""
    nx, ny, nz = (int(s) for s in shape)
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    cube = torch.randn((nx, ny, nz), generator=gen, device=device, dtype=torch.float32)
    if beam_sigma:
        cube = _beam(cube, float(beam_sigma))
    lo, hi = noise_sigma
    if lo != 1.0 or hi != 1.0:
        sig = torch.as_tensor(_noise_sigma_at(np.arange(nz), nz, noise_sigma),
                              dtype=torch.float32, device=device)
        cube *= sig[None, None, :]
    rng = np.random.Generator(np.random.PCG64(int(seed) + 1))
    for _ in range(int(n_sources)):
        cx, cy, cz = rng.uniform(0, nx), rng.uniform(0, ny), rng.uniform(0, nz)
        ss, sf = rng.uniform(1.0, 3.0), rng.uniform(2.0, 10.0)
        amp = rng.uniform(*peak) * float(_noise_sigma_at(cz, nz, noise_sigma))
        x0, x1 = max(0, int(cx - 5 * ss)), min(nx, int(cx + 5 * ss) + 1)
        y0, y1 = max(0, int(cy - 5 * ss)), min(ny, int(cy + 5 * ss) + 1)
        z0, z1 = max(0, int(cz - 5 * sf)), min(nz, int(cz + 5 * sf) + 1)
        if x0 >= x1 or y0 >= y1 or z0 >= z1:
            continue
        ax = torch.arange(x0, x1, device=device, dtype=torch.float64) - cx
        ay = torch.arange(y0, y1, device=device, dtype=torch.float64) - cy
        az = torch.arange(z0, z1, device=device, dtype=torch.float64) - cz
        blob = amp * torch.exp(-(ax[:, None, None] ** 2 + ay[None, :, None] ** 2) / (2 * ss * ss)
                               - az[None, None, :] ** 2 / (2 * sf * sf))
        cube[x0:x1, y0:y1, z0:z1] += blob.to(torch.float32)
    return cube.contiguous()


def make(workload: Workload, device="cpu") -> torch.Tensor:
    """The workload's cube."""
    return make_cube(workload.shape, workload.seed, workload.n_sources, workload.peak,
                     workload.beam_sigma, workload.noise_sigma, device=device)


def subcube_specs(seed: int = 3, n: int = 64, side=(64, 384), length=(128, 2048),
                  sources=(10, 50)) -> list[dict]:
    """Shapes and seeds of the batched workload: n subcubes, Nx = Ny = side.

    side, length and source counts are integer-uniform (inclusive) from PCG64(seed).
    """
    rng = np.random.Generator(np.random.PCG64(int(seed)))
    out = []
    for i in range(int(n)):
        s = int(rng.integers(side[0], side[1] + 1))
        L = int(rng.integers(length[0], length[1] + 1))
        ns = int(rng.integers(sources[0], sources[1] + 1))
        out.append({"shape": (s, s, L), "seed": 1000 * int(seed) + i, "n_sources": ns})
    return out


def make_subcube(spec: dict, device="cpu") -> torch.Tensor:
    """One subcube of the batched workload (noise model of the tile workload)."""
    return make_cube(spec["shape"], spec["seed"], spec["n_sources"], (0.3, 5.0), 1.5,
                     device=device)


def make_weights(shape, seed: int, noise_sigma=(0.8, 1.5), n_flagged: int = 3, flag_width=(4, 24),
                 device="cpu") -> torch.Tensor:
    """Seeded float32 weights cube [x][y][z] for the weighted convolution
    (Eq. 1): inverse noise variance, w = 1 / sigma(z)^2 with sigma rising
    linearly over the channels from noise_sigma[0] to noise_sigma[1] and a
    +-10% smooth spatial ripple, and n_flagged channel ranges (widths
    integer-uniform in flag_width, positions uniform) set to 0, as flagged
    channels are.  Parameters from numpy PCG64(seed + 2)."""
    nx, ny, nz = (int(s) for s in shape)
    rng = np.random.Generator(np.random.PCG64(int(seed) + 2))
    z = np.arange(nz, dtype=np.float64)
    sig = noise_sigma[0] + (noise_sigma[1] - noise_sigma[0]) * z / max(1, nz - 1)
    px, py = rng.uniform(0.0, 2 * math.pi, size=2)
    x = np.arange(nx, dtype=np.float64)[:, None]
    y = np.arange(ny, dtype=np.float64)[None, :]
    ripple = 1.0 + 0.1 * np.sin(2 * math.pi * x / max(8, nx) + px) * np.cos(2 * math.pi * y / max(8, ny) + py)
    w = (ripple[:, :, None] / (sig * sig)[None, None, :]).astype(np.float32)
    for _ in range(int(n_flagged)):
        width = int(rng.integers(flag_width[0], flag_width[1] + 1))
        start = int(rng.integers(0, max(1, nz - width)))
        w[:, :, start:start + width] = 0.0
    return torch.from_numpy(np.ascontiguousarray(w)).to(device)
