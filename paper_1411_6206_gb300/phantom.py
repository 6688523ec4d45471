"""Seeded synthetic inputs for dynamic 3D MRI reconstruction (Priori L+S, arXiv:1411.6206).

This module makes the *inputs* of the method and nothing else: image-domain phantoms,
coil sensitivity maps, variable-density Cartesian masks and complex Gaussian noise. It holds
none of the reconstruction arithmetic (no Fourier encode, no transform, no threshold); the
k-space data d = E(x) + eta is formed by whoever consumes these arrays (the FP64 oracle in
tests, the library's own forward operator in the benchmark).

The paper's dataset (a 256x256x14x20 cardiac cine, Sec. 4) is not available; these phantoms
stand in for it in the same shape family: nz < nx = ny, tens of frames, a smooth low-rank
background plus a beating ellipsoidal "heart", variable-density ky-kz masks that are denser
near the centre of k-space (Sec. 4), the first frame sampled at 50% (Sec. 4, Fig. 2 caption).

Array conventions (shared by every consumer):
  image   complex [nz][nx][ny]           (y fastest)
  coils   complex [ncoil][nz][nx][ny]    sum_c |C_c|^2 = 1 at every voxel
  mask    uint8   [nz][ny]               mask[kz][ky] (3D encode) or mask[z][ky] (per-slice)
  noise   complex [ncoil][m][nx]         m = number of set mask entries, raster order
"""
from __future__ import annotations

import dataclasses
from typing import List

import numpy as np
from scipy import ndimage


@dataclasses.dataclass(frozen=True)
class Workload:
    """One synthetic sequence: volume size, coils, frames, sampling and iteration count."""
    name: str
    nx: int
    ny: int
    nz: int
    ncoil: int
    frames: int
    iters: int
    accel: float            # undersampling factor R of frames >= 2
    seed: int
    phantom: str = "heart"  # "ellipsoids" (two oscillating ellipsoids) or "heart"
    first_frac: float = 0.5  # fraction of lines kept in frame 1
    centre: int = 4          # fully sampled centre is centre x centre (ky, kz) lines
    noise_sigma: float = 1e-3
    fft_z: int = 1           # 1: lines on a (ky, kz) grid; 0: ky lines per slice
    frac_lines: float = 0.0  # if > 0, overrides 1/accel (config "25% of lines")

    @property
    def lines_per_frame(self) -> int:
        n = self.ny * self.nz
        f = self.frac_lines if self.frac_lines > 0 else 1.0 / self.accel
        return int(round(n * f))


# The five workloads of the benchmark specification. Sizes follow the paper's shape family.
SMALL = Workload("plain-32x32x8x8-1coil", 32, 32, 8, 1, 8, 30, 4.0, 1,
                 phantom="ellipsoids", frac_lines=0.25)
CARDIAC = Workload("fp32-128x128x16x20-8coil", 128, 128, 16, 8, 20, 50, 8.0, 2)
PRECISION = Workload("precision-192x192x32x25-12coil", 192, 192, 32, 12, 25, 50, 10.0, 3)
WORKLOADS = {w.name: w for w in (SMALL, CARDIAC, PRECISION)}


def batched_mix(n: int = 64, seed0: int = 400) -> List[Workload]:
    """Uneven problems for the batched variant: in-plane 64..160 step 16, 8..32 slices,
    10..30 frames, 4..16 coils, acceleration 4..12."""
    out = []
    for i in range(n):
        rng = np.random.default_rng(seed0 + i)
        nxy = int(rng.choice(np.arange(64, 161, 16)))
        nz = int(rng.choice([8, 10, 12, 14, 16, 20, 24, 28, 32]))
        frames = int(rng.integers(10, 31))
        ncoil = int(rng.integers(4, 17))
        accel = float(rng.integers(4, 13))
        out.append(Workload(f"mix{i}-{nxy}x{nxy}x{nz}x{frames}-{ncoil}c-R{accel:g}",
                            nxy, nxy, nz, ncoil, frames, 50, accel, seed0 + i))
    return out


def _rng(seed: int, *stream: int) -> np.random.Generator:
    return np.random.default_rng(np.random.SeedSequence([seed, *stream]))


def coil_maps(nx: int, ny: int, nz: int, ncoil: int, seed: int) -> np.ndarray:
    """Smooth complex coil sensitivities normalised to unit sum of squares per voxel.

    A complex white field per coil is Gaussian-smoothed (sigma = n/6 voxels along each axis,
    periodic boundary) and divided by the root sum of squares over coils. A single coil is the
    identity map (the paper's single-coil acquisition)."""
    if ncoil == 1:
        return np.ones((1, nz, nx, ny), np.complex128)
    rng = _rng(seed, 11)
    c = np.empty((ncoil, nz, nx, ny), np.complex128)
    sig = (nz / 6.0, nx / 6.0, ny / 6.0)
    for k in range(ncoil):
        re = rng.standard_normal((nz, nx, ny))
        im = rng.standard_normal((nz, nx, ny))
        c[k] = (ndimage.gaussian_filter(re, sig, mode="wrap")
                + 1j * ndimage.gaussian_filter(im, sig, mode="wrap"))
    sos = np.sqrt(np.sum(np.abs(c) ** 2, axis=0))
    return c / sos[None]


def _grid(nx: int, ny: int, nz: int):
    z = (np.arange(nz) + 0.5) / nz - 0.5
    x = (np.arange(nx) + 0.5) / nx - 0.5
    y = (np.arange(ny) + 0.5) / ny - 0.5
    return np.meshgrid(z, x, y, indexing="ij")


def _ellipsoid(Z, X, Y, c, r):
    return (((Z - c[0]) / r[0]) ** 2 + ((X - c[1]) / r[1]) ** 2
            + ((Y - c[2]) / r[2]) ** 2) <= 1.0


def phantom_sequence(w: Workload) -> np.ndarray:
    """Image sequence [frames][nz][nx][ny], peak magnitude about 1."""
    Z, X, Y = _grid(w.nx, w.ny, w.nz)
    rng = _rng(w.seed, 7)
    T = w.frames
    seq = np.zeros((T, w.nz, w.nx, w.ny), np.complex128)
    if w.phantom == "ellipsoids":
        # Smooth complex background with separable magnitude and phase: Casorati rank 1.
        g = np.exp(-(X ** 2) / (2 * 0.25 ** 2) - (Y ** 2) / (2 * 0.3 ** 2))
        h = 0.6 + 0.4 * np.cos(np.pi * Z)
        ph = np.exp(1j * (1.5 * X + 0.8 * Y + 0.5 * Z))
        bg = 0.4 * g * h * ph
        cents = [(0.05, -0.15, 0.1), (-0.1, 0.2, -0.15)]
        r0 = [(0.3, 0.16, 0.14), (0.25, 0.12, 0.18)]
        amp = [0.85, 0.7 + 0.3 * rng.random()]
        phi = rng.uniform(0, 2 * np.pi, size=2)
        for t in range(T):
            img = bg.copy()
            for k in range(2):
                s = 1.0 + 0.2 * np.sin(2 * np.pi * t / 8.0 + phi[k])
                r = tuple(ri * s for ri in r0[k])
                img[_ellipsoid(Z, X, Y, cents[k], r)] = amp[k]
            seq[t] = img
    else:
        # Background sum_{k<=4} a_k(x,y) b_k(z) c_k(t): rank <= 4 at every t.
        bg_terms = []
        for k in range(4):
            cx, cy = rng.uniform(-0.25, 0.25, 2)
            sx, sy = rng.uniform(0.15, 0.35, 2)
            a = np.exp(-((X - cx) ** 2) / (2 * sx ** 2) - ((Y - cy) ** 2) / (2 * sy ** 2))
            a = a * np.exp(1j * rng.uniform(-2, 2) * (X + Y))
            b = 0.7 + 0.3 * np.cos(np.pi * (k + 1) * Z + rng.uniform(0, np.pi))
            bg_terms.append((0.25 * a * b, rng.uniform(0, 2 * np.pi), 0.05 + 0.05 * rng.random()))
        # Beating heart: blood pool (bright) inside a myocardium shell; radii oscillate.
        cen = (0.0, 0.05, -0.03)
        r_in0 = (0.40, 0.20, 0.19)
        r_out0 = (0.46, 0.26, 0.25)
        beat = 8.0
        amp = 0.26
        for t in range(T):
            img = np.zeros_like(Z, dtype=np.complex128)
            for (ab, ph0, ca) in bg_terms:
                img += ab * (1.0 + ca * np.sin(2 * np.pi * t / T + ph0))
            s = 1.0 + amp * np.sin(2 * np.pi * t / beat)
            r_out = tuple(r * (1.0 + 0.5 * (s - 1.0)) for r in r_out0)
            r_in = tuple(r * s for r in r_in0)
            myo = _ellipsoid(Z, X, Y, cen, r_out)
            pool = _ellipsoid(Z, X, Y, cen, r_in)
            img[myo] = 0.55 * np.exp(0.3j)
            img[pool] = 1.0
            seq[t] = img
    return seq


def changed_fraction(seq: np.ndarray, tol: float = 0.05) -> float:
    """Mean fraction of voxels whose value moves by more than `tol` between frames."""
    if seq.shape[0] < 2:
        return 0.0
    d = np.abs(np.diff(seq, axis=0)) > tol
    return float(d.mean())


def _signed(n: int) -> np.ndarray:
    k = np.arange(n)
    return np.where(k < (n + 1) // 2, k, k - n)


def vd_mask(ny: int, nz: int, n_lines: int, centre: int, seed: int, fft_z: int = 1) -> np.ndarray:
    """Variable-density Cartesian mask [nz][ny] (uint8), unshifted DFT index order.

    fft_z=1: n_lines entries of the (ky, kz) grid, a centre x centre block of the lowest
    signed frequencies always kept, the rest drawn without replacement with weight
    (1 - rho)^2, rho the normalised radius in signed-frequency space.
    fft_z=0: per slice z, round(n_lines / nz) ky lines with `centre` centre lines kept."""
    rng = _rng(seed, 3)
    m = np.zeros((nz, ny), np.uint8)
    ky = _signed(ny)
    if fft_z:
        kz = _signed(nz)
        KZ, KY = np.meshgrid(kz, ky, indexing="ij")
        h = centre // 2
        core = (KY >= -h) & (KY < centre - h) & (KZ >= -h) & (KZ < centre - h)
        m[core] = 1
        rho = np.sqrt((KY / (ny / 2.0)) ** 2 + (KZ / (nz / 2.0)) ** 2) / np.sqrt(2.0)
        w = np.clip(1.0 - rho, 0.0, None) ** 2
        w[core] = 0.0
        need = int(n_lines) - int(core.sum())
        cand = np.flatnonzero(w.ravel() > 0)
        need = max(0, min(need, cand.size))
        p = w.ravel()[cand]
        pick = rng.choice(cand, size=need, replace=False, p=p / p.sum())
        m.ravel()[pick] = 1
    else:
        per = max(centre, int(round(n_lines / nz)))
        h = centre // 2
        core = (ky >= -h) & (ky < centre - h)
        rho = np.abs(ky) / (ny / 2.0)
        w = np.clip(1.0 - rho, 0.0, None) ** 2
        w[core] = 0.0
        cand = np.flatnonzero(w > 0)
        for z in range(nz):
            m[z, core] = 1
            need = max(0, min(per - int(core.sum()), cand.size))
            p = w[cand]
            pick = rng.choice(cand, size=need, replace=False, p=p / p.sum())
            m[z, pick] = 1
    return m


def noise(ncoil: int, m: int, nx: int, sigma: float, seed: int) -> np.ndarray:
    """CN(0, sigma^2) samples [ncoil][m][nx]: real and imaginary parts each N(0, sigma^2/2)."""
    rng = _rng(seed, 5)
    s = sigma / np.sqrt(2.0)
    return s * (rng.standard_normal((ncoil, m, nx)) + 1j * rng.standard_normal((ncoil, m, nx)))


def masks_for(w: Workload) -> List[np.ndarray]:
    out = []
    for t in range(w.frames):
        frac = w.first_frac if t == 0 else None
        n = int(round(w.ny * w.nz * frac)) if frac else w.lines_per_frame
        out.append(vd_mask(w.ny, w.nz, n, w.centre, w.seed * 1000 + t, w.fft_z))
    return out


def problem(w: Workload, frames: int | None = None):
    """Everything a reconstruction of `w` consumes, except the k-space data itself.

    Returns dict(x=[T][nz][nx][ny], coils, masks=[T][nz][ny], noise=[T][ncoil][m_t][nx])."""
    T = w.frames if frames is None else min(frames, w.frames)
    x = phantom_sequence(w)[:T]
    coils = coil_maps(w.nx, w.ny, w.nz, w.ncoil, w.seed)
    masks = masks_for(w)[:T]
    nz_ = [noise(w.ncoil, int(mk.sum()), w.nx, w.noise_sigma, w.seed * 1000 + t)
           for t, mk in enumerate(masks)]
    return dict(x=x, coils=coils, masks=masks, noise=nz_)
