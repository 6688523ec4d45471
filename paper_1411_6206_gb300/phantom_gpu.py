"""Device-side versions of the seeded input generators, for workloads too large to generate
on the host in a benchmark run (the batched and serving mixes). Same recipes as phantom.py:

- coil maps: complex white fields, Gaussian-smoothed with sigma = n/6 voxels per axis under a
  periodic boundary (here by the Gaussian's transfer function in the Fourier domain), divided
  by the root sum of squares over coils; one coil is the identity map;
- frames: the beating-heart family (rank <= 4 smooth background whose weights drift over the
  sequence, a bright blood pool inside a myocardium shell whose radii oscillate with a period
  of 8 frames); the background parameters are drawn from the same seeded generator as the
  host version;
- noise: CN(0, sigma^2) per k-space sample.

Values differ from phantom.py at the level of the smoothing kernel and the random streams;
the shapes, value ranges and structure are the same. Nothing here computes any part of the
reconstruction.
"""
from __future__ import annotations

import math

import numpy as np

from . import phantom as P


def coil_maps(nx: int, ny: int, nz: int, ncoil: int, seed: int, device="cuda"):
    import torch
    if ncoil == 1:
        return torch.ones((1, nz, nx, ny), dtype=torch.complex64, device=device)
    g = torch.Generator(device=device).manual_seed(int(seed))
    c = torch.complex(torch.randn((ncoil, nz, nx, ny), generator=g, device=device),
                      torch.randn((ncoil, nz, nx, ny), generator=g, device=device))
    # Gaussian blur (sigma_axis = n_axis / 6 voxels), periodic: multiply the spectrum by
    # exp(-2 pi^2 sigma^2 f^2) with f in cycles per voxel
    filt = torch.ones((nz, nx, ny), device=device)
    for ax, n in enumerate((nz, nx, ny)):
        f = torch.fft.fftfreq(n, device=device)
        h = torch.exp(-2.0 * math.pi ** 2 * (n / 6.0) ** 2 * f ** 2)
        shape = [1, 1, 1]
        shape[ax] = n
        filt = filt * h.reshape(shape)
    c = torch.fft.ifftn(torch.fft.fftn(c, dim=(1, 2, 3)) * filt, dim=(1, 2, 3))
    sos = torch.sqrt((c.abs() ** 2).sum(0, keepdim=True))
    return (c / sos).to(torch.complex64).contiguous()


class HeartFrames:
    """Frame generator of the beating-heart family on the device: frame(t) -> [nz][nx][ny]."""

    def __init__(self, w: P.Workload, device="cuda"):
        import torch
        self.w = w
        self.device = device
        z = (torch.arange(w.nz, device=device, dtype=torch.float64) + 0.5) / w.nz - 0.5
        x = (torch.arange(w.nx, device=device, dtype=torch.float64) + 0.5) / w.nx - 0.5
        y = (torch.arange(w.ny, device=device, dtype=torch.float64) + 0.5) / w.ny - 0.5
        self.Z, self.X, self.Y = torch.meshgrid(z, x, y, indexing="ij")
        rng = P._rng(w.seed, 7)
        self.bg = []
        for k in range(4):
            cx, cy = rng.uniform(-0.25, 0.25, 2)
            sx, sy = rng.uniform(0.15, 0.35, 2)
            a = torch.exp(-((self.X - cx) ** 2) / (2 * sx ** 2) - ((self.Y - cy) ** 2) / (2 * sy ** 2))
            a = a * torch.exp(1j * float(rng.uniform(-2, 2)) * (self.X + self.Y))
            b = 0.7 + 0.3 * torch.cos(math.pi * (k + 1) * self.Z + float(rng.uniform(0, np.pi)))
            self.bg.append((0.25 * a * b, float(rng.uniform(0, 2 * np.pi)), 0.05 + 0.05 * float(rng.random())))

    def _ell(self, c, r):
        return (((self.Z - c[0]) / r[0]) ** 2 + ((self.X - c[1]) / r[1]) ** 2 + ((self.Y - c[2]) / r[2]) ** 2) <= 1.0

    def frame(self, t: int):
        import torch
        T = self.w.frames
        img = torch.zeros_like(self.Z, dtype=torch.complex128)
        for ab, ph0, ca in self.bg:
            img = img + ab * (1.0 + ca * math.sin(2 * math.pi * t / T + ph0))
        s = 1.0 + 0.26 * math.sin(2 * math.pi * t / 8.0)
        cen = (0.0, 0.05, -0.03)
        r_out = tuple(r * (1.0 + 0.5 * (s - 1.0)) for r in (0.46, 0.26, 0.25))
        r_in = tuple(r * s for r in (0.40, 0.20, 0.19))
        img[self._ell(cen, r_out)] = 0.55 * complex(math.cos(0.3), math.sin(0.3))
        img[self._ell(cen, r_in)] = 1.0
        return img.to(torch.complex64).contiguous()


def noise(ncoil: int, m: int, nx: int, sigma: float, seed: int, device="cuda"):
    import torch
    g = torch.Generator(device=device).manual_seed(int(seed))
    s = sigma / math.sqrt(2.0)
    return torch.complex(s * torch.randn((ncoil, m, nx), generator=g, device=device),
                         s * torch.randn((ncoil, m, nx), generator=g, device=device))
