"""Test-side helpers: the C ABI's wavelet-coefficient order versus the oracle's Mallat layout.

The ABI numbers the coefficients of slice z tile by tile (8 x 8 in-plane tiles); inside a
tile every aligned 2^J x 2^J sub-block keeps its own Mallat layout (lps_api.h); with the 3D
transform the slices of every aligned 2^J-slice block hold that block's 1D Mallat layout along
z as well. The oracle stores the whole-plane (whole-volume) Mallat pyramid. Both are orderings of the same orthonormal Haar
coefficients; this module maps one to the other so bitmaps can be compared.
"""
import numpy as np


def _mallat_1d(n: int, B: int, blk: int, w: int) -> int:
    """Whole-axis Mallat position of in-block position w of aligned block blk (block B)."""
    if w == 0:
        return blk
    h = 1 << (w.bit_length() - 1)
    return n * h // B + blk * h + (w - h)


def abi_to_mallat(nz: int, nx: int, ny: int, J: int, dims: int = 2):
    """Arrays (z, i, j) of Mallat positions, indexed by the ABI coefficient index."""
    B = 1 << J
    ntx, nty = nx // 8, ny // 8
    n = nz * nx * ny
    zz = np.empty(n, np.int64)
    ii = np.empty(n, np.int64)
    jj = np.empty(n, np.int64)
    k = 0
    for z in range(nz):
        for tx in range(ntx):
            for ty in range(nty):
                for u in range(8):
                    for v in range(8):
                        su, sv = u // B, v // B
                        up, vp = u % B, v % B
                        bx, by = tx * (8 // B) + su, ty * (8 // B) + sv
                        if up == 0 and vp == 0:
                            i, j = bx, by
                        else:
                            m = max(up, vp)
                            h = 1 << (m.bit_length() - 1)
                            ox, oy = nx * h // B, ny * h // B
                            if up < h:
                                i, j = bx * h + up, oy + by * h + (vp - h)
                            elif vp < h:
                                i, j = ox + bx * h + (up - h), by * h + vp
                            else:
                                i, j = ox + bx * h + (up - h), oy + by * h + (vp - h)
                        zm = z if dims == 2 else _mallat_1d(nz, B, z // B, z % B)
                        zz[k], ii[k], jj[k] = zm, i, j
                        k += 1
    return zz, ii, jj


def bits_to_mallat(words: np.ndarray, nz: int, nx: int, ny: int, J: int, dims: int = 2) -> np.ndarray:
    """Unpack an ABI bitmap (uint32 words) into a bool array in Mallat layout [nz][nx][ny]."""
    w = np.asarray(words, np.uint32)
    bits = ((w[:, None] >> np.arange(32, dtype=np.uint32)[None, :]) & 1).astype(bool).ravel()
    zz, ii, jj = abi_to_mallat(nz, nx, ny, J, dims)
    out = np.zeros((nz, nx, ny), bool)
    out[zz, ii, jj] = bits[: zz.size]
    return out


def mallat_to_bits(sup: np.ndarray, J: int, dims: int = 2) -> np.ndarray:
    """Pack a bool Mallat-layout support [nz][nx][ny] into ABI uint32 words."""
    nz, nx, ny = sup.shape
    zz, ii, jj = abi_to_mallat(nz, nx, ny, J, dims)
    b = sup[zz, ii, jj].astype(np.uint32).reshape(-1, 32)
    return (b << np.arange(32, dtype=np.uint32)[None, :]).sum(axis=1).astype(np.uint32)


def mallat_to_abi_values(c: np.ndarray, J: int, dims: int = 2) -> np.ndarray:
    nz, nx, ny = c.shape
    zz, ii, jj = abi_to_mallat(nz, nx, ny, J, dims)
    return c[zz, ii, jj]
