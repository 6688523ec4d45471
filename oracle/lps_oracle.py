"""FP64 CPU oracle for Priori L+S (Zonoobi, Faghih Roohi, Kassim, arXiv:1411.6206).

TEST INFRASTRUCTURE ONLY. This module is imported by the tests, by the smoke check and by
the benchmark's CPU-baseline leg. The library's product path never imports, calls or links
it, and it shares no code with the CUDA path.

Every function computes the plain definition in float64 / complex128, with no blocking,
fusion or algebraic shortcut beyond what the definition states:

  E, E^H      acquisition operator of Sec. 2 (d = A(X) + eta, A^{-1} denotes the adjoint per
              the notation paragraph of Sec. 1), extended to multiple receive coils:
              E x = M F (C_c x) for every coil c, F the orthonormal unshifted DFT over
              (z, x, y) (or over (x, y) per slice), M the Cartesian line mask.
              Implemented with scipy.fft.fftn(norm="ortho") on the full grid.
  T, T^{-1}   the sparsifying transform of Sec. 2 ("Wavelets"; Sec. 4 "Wavelet domain"):
              orthonormal 2D Haar, Mallat pyramid, J levels, per slice, explicit filter bank;
              T3 the 3D variant (the same per slice, then J levels of the 1D Haar along z).
  soft        the soft-threshold operator of Sec. 2 (x/|x| max(|x|-lambda, 0), complex x).
  svt         singular-value soft-thresholding, Algorithm 1 step (1), via numpy.linalg.svd
              of the Casorati matrix (no Gram-matrix route).
  priori_ls   Algorithm 1 steps (0)-(4) in the paper's order and notation.
  sequence    the recursion over time instances of Sec. 3 (plain L+S at t=1, Algorithm 1
              with the priors of t-1 afterwards; Fig. 2).

Readings of passages that are silent, ambiguous or garbled (each is listed with its reason
in the design document of this repository):
  R1 Casorati columns are the nz slices of one volume (Sec. 2): M in C^{(nx ny) x nz}; the
     "frames" layout takes columns of frame_slices consecutive slices (3D frame volumes, each
     with its own 3D encode and mask) instead.
  R2 lambda_L = lambda_L_rel * sigma_max(X_0), lambda_S = lambda_S_rel * max|T(X_0)|,
     fixed once per frame (the paper gives no values; lambda_T in the input list of
     Algorithm 1 is read as lambda_L).
  R3 Step (3) shrinks T(X_{it-1} - L_{it-1}) with L_0 := X_0 (Otazo's L+S ordering; the
     literal T(S_{it-1}) with S_0 = 0 would keep S at zero forever).
  R4 Step (4) uses X = L + S - E^H(E(L + S) - d) (descent; the printed sign of E_it is
     the ascent direction and diverges).
  R5 T^(t) = {i : |c_i| > lambda_S} for c of the final iteration (threshold support
     detection); ties at lambda_S are off-support. The literal nonzero rule is optional.
  R6 T = orthonormal 2D Haar (Mallat), J = 3, every coefficient thresholded.
  R7 singular values are matched to sigma_prev by rank (both descending); directions with
     sigma_i <= tau * sigma_1 are dropped after step (2) (rank guard).
  R8 soft(0, lambda) = 0; |x| = lambda gives 0.
  R9 the 3D variant of T (wavelet_dims = 3) is the tensor product of the 2D pyramid of R6
     with the J-level 1D Haar along z; nz a multiple of 2^J.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional

import numpy as np
import scipy.fft as sfft


# ----------------------------------------------------------------------------------------
# Acquisition operator (Sec. 2) and its adjoint
# ----------------------------------------------------------------------------------------

def line_index(mask: np.ndarray):
    """Sampled lines of a [nz][ny] mask in raster order: (first index, ky) pairs."""
    flat = np.flatnonzero(np.asarray(mask).ravel())
    ny = mask.shape[1]
    return flat // ny, flat % ny


def _axes(fft_z: int):
    return (0, 1, 2) if fft_z else (1, 2)


def _fft(a: np.ndarray, fft_z: int, zblock: Optional[int], inverse: bool) -> np.ndarray:
    """Orthonormal DFT over (z, x, y) of an image [nz][nx][ny]: over all nz slices (fft_z = 1),
    per slice (fft_z = 0), or over each aligned block of `zblock` slices separately (the 3D
    encode of every frame volume when the Casorati columns are volumes of zblock slices)."""
    f = sfft.ifftn if inverse else sfft.fftn
    if zblock is None or zblock == a.shape[0]:
        return f(a, axes=_axes(fft_z), norm="ortho")
    nz, nx, ny = a.shape
    blocks = a.reshape(nz // zblock, zblock, nx, ny)
    return f(blocks, axes=(1, 2, 3), norm="ortho").reshape(nz, nx, ny)


def E(x: np.ndarray, coils: np.ndarray, mask: np.ndarray, fft_z: int = 1,
      zblock: Optional[int] = None) -> np.ndarray:
    """d = M F (C x): image [nz][nx][ny] -> samples [ncoil][m][nx] (Sec. 2, acquisition)."""
    kz, ky = line_index(mask)
    ncoil = coils.shape[0]
    out = np.empty((ncoil, kz.size, x.shape[1]), np.complex128)
    for c in range(ncoil):
        K = _fft(coils[c] * x, fft_z, zblock, False)
        out[c] = K[kz, :, ky]
    return out


def EH(d: np.ndarray, coils: np.ndarray, mask: np.ndarray, fft_z: int = 1,
       zblock: Optional[int] = None) -> np.ndarray:
    """x = sum_c conj(C_c) F^H M^T d_c: samples [ncoil][m][nx] -> image [nz][nx][ny]."""
    kz, ky = line_index(mask)
    ncoil, nz, nx, ny = coils.shape
    x = np.zeros((nz, nx, ny), np.complex128)
    for c in range(ncoil):
        K = np.zeros((nz, nx, ny), np.complex128)
        K[kz, :, ky] = d[c]
        x += np.conj(coils[c]) * _fft(K, fft_z, zblock, True)
    return x


# ----------------------------------------------------------------------------------------
# Sparsifying transform T: orthonormal Haar, Mallat pyramid, per slice (Sec. 2 / Sec. 4)
# ----------------------------------------------------------------------------------------

_R2 = 1.0 / np.sqrt(2.0)


def _haar_split(a: np.ndarray, axis: int):
    ev = np.take(a, np.arange(0, a.shape[axis], 2), axis=axis)
    od = np.take(a, np.arange(1, a.shape[axis], 2), axis=axis)
    return (ev + od) * _R2, (ev - od) * _R2


def _haar_merge(lo: np.ndarray, hi: np.ndarray, axis: int):
    shape = list(lo.shape)
    shape[axis] *= 2
    out = np.empty(shape, np.result_type(lo, hi))
    ev = (lo + hi) * _R2
    od = (lo - hi) * _R2
    idx_e = [slice(None)] * lo.ndim
    idx_o = [slice(None)] * lo.ndim
    idx_e[axis] = slice(0, None, 2)
    idx_o[axis] = slice(1, None, 2)
    out[tuple(idx_e)] = ev
    out[tuple(idx_o)] = od
    return out


def haar2(plane: np.ndarray, J: int) -> np.ndarray:
    """J-level 2D orthonormal Haar of a [nx][ny] plane in Mallat layout.

    At each level the current approximation block [:hx, :hy] is split along y (axis 1) and
    then along x (axis 0); the four sub-bands are stored as
      [:hx/2, :hy/2]  approximation      [:hx/2, hy/2:hy]  x-low / y-high
      [hx/2:hx, :hy/2] x-high / y-low    [hx/2:hx, hy/2:hy] x-high / y-high."""
    out = np.array(plane, dtype=np.complex128, copy=True)
    hx, hy = out.shape
    for _ in range(J):
        blk = out[:hx, :hy]
        ylo, yhi = _haar_split(blk, 1)
        ll, hl = _haar_split(ylo, 0)
        lh, hh = _haar_split(yhi, 0)
        out[:hx // 2, :hy // 2] = ll
        out[:hx // 2, hy // 2:hy] = lh
        out[hx // 2:hx, :hy // 2] = hl
        out[hx // 2:hx, hy // 2:hy] = hh
        hx //= 2
        hy //= 2
    return out


def ihaar2(coef: np.ndarray, J: int) -> np.ndarray:
    """Inverse of haar2."""
    out = np.array(coef, dtype=np.complex128, copy=True)
    nx, ny = out.shape
    hx, hy = nx >> (J - 1), ny >> (J - 1)
    for _ in range(J):
        ll = out[:hx // 2, :hy // 2]
        lh = out[:hx // 2, hy // 2:hy]
        hl = out[hx // 2:hx, :hy // 2]
        hh = out[hx // 2:hx, hy // 2:hy]
        ylo = _haar_merge(ll, hl, 0)
        yhi = _haar_merge(lh, hh, 0)
        out[:hx, :hy] = _haar_merge(ylo, yhi, 1)
        hx *= 2
        hy *= 2
    return out


def T(x: np.ndarray, J: int = 3) -> np.ndarray:
    """Haar coefficients of every slice of an image [nz][nx][ny] (same shape, Mallat)."""
    return np.stack([haar2(x[z], J) for z in range(x.shape[0])])


def Tinv(c: np.ndarray, J: int = 3) -> np.ndarray:
    return np.stack([ihaar2(c[z], J) for z in range(c.shape[0])])


def T3(x: np.ndarray, J: int = 3) -> np.ndarray:
    """3D orthonormal Haar (the tensor-product variant): the per-slice 2D transform T, then J
    levels of the 1D Haar along z over the whole nz in Mallat order (at each level the leading
    approximation block is split into low and high halves). nz must be a multiple of 2^J."""
    out = np.array(T(x, J), dtype=np.complex128, copy=True)
    hz = out.shape[0]
    for _ in range(J):
        lo, hi = _haar_split(out[:hz], 0)
        out[:hz // 2] = lo
        out[hz // 2:hz] = hi
        hz //= 2
    return out


def T3inv(c: np.ndarray, J: int = 3) -> np.ndarray:
    out = np.array(c, dtype=np.complex128, copy=True)
    hz = out.shape[0] >> (J - 1)
    for _ in range(J):
        out[:hz] = _haar_merge(out[:hz // 2], out[hz // 2:hz], 0)
        hz *= 2
    return Tinv(out, J)


def sparsifying(p):
    """The transform pair of step (3): T (2D per slice, the default) or T3 (3D)."""
    return (T3, T3inv) if p.wavelet_dims == 3 else (T, Tinv)


# ----------------------------------------------------------------------------------------
# Pointwise and singular-value operators
# ----------------------------------------------------------------------------------------

def soft(x: np.ndarray, lam: float) -> np.ndarray:
    """Soft threshold of Sec. 2: x/|x| * max(|x| - lam, 0), with 0 at x = 0 (R8)."""
    x = np.asarray(x)
    a = np.abs(x)
    scale = np.where(a > lam, (a - lam) / np.where(a > 0, a, 1.0), 0.0)
    return x * scale


def casorati(x: np.ndarray, cs: int = 1) -> np.ndarray:
    """[nz][nx][ny] -> Casorati matrix [(cs nx ny)][nz / cs]: one column per slice (R1), or,
    with cs > 1, per volume of cs consecutive slices (the "frames" layout of 3D frames)."""
    nz = x.shape[0]
    return x.reshape(nz // cs, -1).T


def uncasorati(m: np.ndarray, shape) -> np.ndarray:
    return m.T.reshape(shape)


def casorati_gram(X: np.ndarray, S: Optional[np.ndarray] = None, cs: int = 1) -> np.ndarray:
    """G = M^H M of the Casorati matrix M = casorati(X - S): the small Hermitian matrix
    whose eigenpairs are the squared singular values and right singular vectors that the
    singular-value thresholding of step (1) (Sec. 3) acts on. Plain definition, FP64."""
    M = casorati(X if S is None else X - S, cs).astype(np.complex128)
    return M.conj().T @ M


def reproject(X: np.ndarray, S: Optional[np.ndarray], W: np.ndarray, cs: int = 1) -> np.ndarray:
    """L = uncasorati((X - S) W): with W = V diag(sigma''/sigma) V^H this is the low-rank
    term U diag(sigma'') V^H of steps (1)-(2) (Sec. 3). Plain definition, FP64."""
    M = casorati(X if S is None else X - S, cs).astype(np.complex128)
    return uncasorati(M @ np.asarray(W, np.complex128), X.shape)


def svt(mat: np.ndarray, lam_L: float, lam_p: float = 0.0,
        sigma_prev: Optional[np.ndarray] = None, tau: float = 0.0):
    """Steps (1)-(2) of Algorithm 1 on a Casorati matrix.

    sigma' = max(sigma - lam_L, 0)                      step (1)
    sigma'' = sigma' - lam_p (sigma' - sigma_prev)      step (2), rank-matched (R7)
    sigma''_i = 0 where sigma_i <= tau sigma_1          rank guard (R7)
    Returns (L = U diag(sigma'') V^H, sigma, sigma'')."""
    U, s, Vh = np.linalg.svd(mat, full_matrices=False)
    s1 = np.maximum(s - lam_L, 0.0)
    if sigma_prev is not None:
        s2 = s1 - lam_p * (s1 - np.asarray(sigma_prev, np.float64))
    else:
        s2 = s1
    s2 = np.where(s <= tau * s[0], 0.0, s2) if s.size else s2
    L = (U * s2[None, :]) @ Vh
    return L, s, s2


def support_shrink(c: np.ndarray, lam_S: float, keep: Optional[np.ndarray]) -> np.ndarray:
    """Step (3): coefficients on the prior support are kept, the rest soft-thresholded."""
    sh = soft(c, lam_S)
    if keep is None:
        return sh
    return np.where(keep, c, sh)


# ----------------------------------------------------------------------------------------
# Algorithm 1 and the recursion over t
# ----------------------------------------------------------------------------------------

@dataclasses.dataclass
class Params:
    lambda_L_rel: float = 0.01
    lambda_S_rel: float = 0.005
    lambda_p: float = 0.5
    rank_tau: float = 1e-3
    wavelet_levels: int = 3
    max_iters: int = 50
    tol: float = 0.0
    fft_z: int = 1
    support_rule: str = "threshold"   # or "nonzero"
    wavelet_dims: int = 2             # 2: per-slice 2D Haar (R6); 3: 3D tensor-product Haar
    frame_slices: int = 1             # slices per Casorati column (> 1: columns are 3D frames)


@dataclasses.dataclass
class Result:
    L: np.ndarray
    S: np.ndarray
    support: np.ndarray       # bool, Mallat layout [nz][nx][ny]
    sigma: np.ndarray         # sigma'' of the last iteration, rank order
    lambda_L: float
    lambda_S: float
    iters: int
    history: list             # per iteration: dict(resid2, nuclear, l1, objective, rel_change)
    X: np.ndarray             # X of the last iteration (step 4 output)
    c: np.ndarray             # T(X_{K-1} - L_{K-1}) of the last iteration
    sigma_in: np.ndarray = None   # singular values of X - S entering the last step (1)

    @property
    def recon(self):
        return self.L + self.S


@dataclasses.dataclass
class Prior:
    support: Optional[np.ndarray] = None   # bool [nz][nx][ny], Mallat layout
    sigma: Optional[np.ndarray] = None     # sigma'' of the previous frame, rank order


def zblock_of(p: Params) -> Optional[int]:
    """Slices per z transform of E: each frame volume alone when the columns are 3D frames
    (its slices with the 3D encode, one at a time without it), else the fft_z default."""
    if p.frame_slices > 1:
        return p.frame_slices if p.fft_z else 1
    return None


def initial_lambdas(X0: np.ndarray, p: Params):
    s = np.linalg.svd(casorati(X0, p.frame_slices), compute_uv=False)
    Tf, _ = sparsifying(p)
    return p.lambda_L_rel * s[0], p.lambda_S_rel * np.max(np.abs(Tf(X0, p.wavelet_levels)))


def priori_ls(d, coils, mask, p: Params, prior: Optional[Prior] = None,
              iters: Optional[int] = None, state=None) -> Result:
    """Algorithm 1 (PrioriL+S decomposition) for one time instance.

    d      samples [ncoil][m][nx];  coils [ncoil][nz][nx][ny];  mask [nz][ny]
    prior  None (t = 1, plain L+S) or Prior(support, sigma) of frame t-1
    state  optional (X, S, L_prev, lambda_L, lambda_S) to start from instead of step (0)."""
    J = p.wavelet_levels
    Tf, Tfinv = sparsifying(p)
    K = p.max_iters if iters is None else iters
    zb, cs = zblock_of(p), p.frame_slices
    if state is None:
        X = EH(d, coils, mask, p.fft_z, zb)           # (0) X_0 = A^{-1}(y)
        S = np.zeros_like(X)                          #     S_0 = 0
        Lp = X.copy()                                 #     L_0 := X_0 (R3)
        lamL, lamS = initial_lambdas(X, p)            # R2
    else:
        X, S, Lp, lamL, lamS = (np.array(state[0], np.complex128), np.array(state[1], np.complex128),
                                np.array(state[2], np.complex128), float(state[3]), float(state[4]))
    keep = None
    sig_prev = None
    if prior is not None:
        keep = prior.support
        sig_prev = prior.sigma
    shape = X.shape
    hist = []
    c = np.zeros_like(X)
    it = 0
    L = Lp
    s2 = np.zeros(shape[0] // cs)
    s = np.zeros(shape[0] // cs)
    for it in range(1, K + 1):
        Z_old = Lp + S
        # (1) singular-value soft-thresholding of X_{it-1} - S_{it-1}
        # (2) prior pull of the singular values towards those of L^(t-1)
        Lm, s, s2 = svt(casorati(X - S, cs), lamL, p.lambda_p, sig_prev, p.rank_tau)
        L = uncasorati(Lm, shape)
        # (3) sparsity off the prior support
        c = Tf(X - Lp, J)
        c2 = support_shrink(c, lamS, keep)
        S = Tfinv(c2, J)
        # (4) data consistency
        R = E(L + S, coils, mask, p.fft_z, zb) - d
        X = L + S - EH(R, coils, mask, p.fft_z, zb)
        Lp = L
        resid2 = float(np.vdot(R, R).real)
        off = np.ones(c.shape, bool) if keep is None else ~keep
        l1 = float(np.abs(c2[off]).sum())
        nuc = float(s2.sum())
        Z = L + S
        rel = float(np.linalg.norm(Z - Z_old) / max(np.linalg.norm(Z_old), 1e-300))
        hist.append(dict(resid2=resid2, nuclear=nuc, l1=l1,
                         objective=0.5 * resid2 + lamL * nuc + lamS * l1, rel_change=rel))
        if p.tol > 0 and rel < p.tol:
            break
    if p.support_rule == "nonzero":
        sup = support_shrink(c, lamS, keep) != 0
    else:
        sup = np.abs(c) > lamS
    return Result(L=L, S=S, support=sup, sigma=np.array(s2, np.float64), lambda_L=lamL,
                  lambda_S=lamS, iters=it, history=hist, X=X, c=c, sigma_in=np.array(s, np.float64))


def objective(L, S, d, coils, mask, lamL, lamS, keep, p: Params) -> float:
    """F(L, S) = 1/2 ||E(L + S) - d||^2 + lamL ||L||_* + lamS ||T(S)|_{off prior}||_1,
    the Lagrangian form of Eq. (3) without the sigma-closeness constraint (lambda_p = 0)."""
    R = E(L + S, coils, mask, p.fft_z, zblock_of(p)) - d
    nuc = np.linalg.svd(casorati(L, p.frame_slices), compute_uv=False).sum()
    c = sparsifying(p)[0](S, p.wavelet_levels)
    off = np.ones(c.shape, bool) if keep is None else ~keep
    return 0.5 * float(np.vdot(R, R).real) + lamL * nuc + lamS * float(np.abs(c[off]).sum())


def sequence(datas: List[np.ndarray], coils, masks, p: Params, frames: Optional[int] = None):
    """Recursion over time (Sec. 3, Fig. 2): t = 1 is plain L+S, later frames use the
    support and singular values of the previous reconstruction as priors."""
    out = []
    prior = None
    T_ = len(datas) if frames is None else frames
    for t in range(T_):
        r = priori_ls(datas[t], coils, masks[t], p, prior)
        out.append(r)
        prior = Prior(support=r.support, sigma=r.sigma)
    return out


def nrmse(a: np.ndarray, ref: np.ndarray) -> float:
    return float(np.linalg.norm(a - ref) / max(np.linalg.norm(ref), 1e-300))


def psnr(a: np.ndarray, ref: np.ndarray) -> float:
    mse = float(np.mean(np.abs(a - ref) ** 2))
    return float(10 * np.log10(np.max(np.abs(ref)) ** 2 / max(mse, 1e-300)))
