"""Streaming reconstruction of a 2D + time sequence with a sliding temporal window.

The Casorati matrix is voxels x the last W frames (layout "frames": column z is frame
t - W + 1 + z, each with its own ky lines and 2D encode). Every new frame advances the window by
one and reconstructs it with Algorithm 1 (Sec. 3); the recursion of Sec. 3 carries the support
and the singular values of the previous window, the support moved one column so that every
frame keeps its own (the newest frame takes the support of the frame before it), and the
eigenvectors of the previous window's Gram start the next eigendecomposition. The newest frame
of each window (column W - 1 of L + S) is the stream's output.

This module orders calls and keeps the rings of per-frame masks and samples; it holds none of
the method's arithmetic.
"""
from __future__ import annotations

from collections import deque

import numpy as np


class SlidingWindow:
    def __init__(self, lps, nx: int, ny: int, ncoil: int, window: int, coils, stream=None, **params):
        """coils: complex64 [ncoil][nx][ny] maps of the slice (device tensor), the same for every
        frame; params: further lps_params fields (iterations, lambdas, ...)."""
        import torch
        self.lps = lps
        self.nx, self.ny, self.ncoil, self.W = nx, ny, ncoil, window
        self.plan = lps.Plan(nx, ny, window, ncoil, stream=stream, layout=lps.LAYOUT_FRAMES, fft_z=0, recursive=1,
                             **params)
        self.plan.set_coils(coils[:, None].expand(ncoil, window, nx, ny).contiguous())
        self.masks = deque(maxlen=window)
        self.data = deque(maxlen=window)
        self.windows = 0
        self.recon = torch.empty((window, nx, ny), dtype=torch.complex64, device=coils.device)

    def push(self, mask_row, samples):
        """Add frame t: its sampled ky lines (uint8 [ny], host) and samples (complex64
        [ncoil][lines][nx], device). Returns the reconstruction of frame t (a view of the
        window's last column) once W frames have arrived, else None."""
        import torch
        self.masks.append(np.asarray(mask_row, np.uint8))
        self.data.append(samples)
        if len(self.masks) < self.W:
            return None
        if self.windows:
            self.lps.shift_prior_columns(self.plan.handle, 1)
        mask = np.ascontiguousarray(np.stack(list(self.masks)))
        n = self.plan.set_mask(mask)
        d = torch.cat(list(self.data), dim=1)
        assert d.shape[1] == n
        self.plan.set_data(d.contiguous())
        self.plan.reconstruct_frame(recon=self.recon, stats=False)
        self.windows += 1
        return self.recon[self.W - 1]

    def close(self):
        self.plan.close()
