"""One x-slab of the FP64 oracle's Algorithm 1: test infrastructure for the x-slab sharding.

A slab holds planes x0 .. x0+nx-1 of a volume of nx_total planes and runs the steps of
Algorithm 1 (Sec. 3) in the oracle's order with the oracle's operators restricted to its
planes. With F the orthonormal DFT over (z, x, y) = F_x (x) F_zy, the samples moved along kx
to the hybrid space, d'_c = F_x^H d_c, restrict per plane: E_slab Z = M F_zy (C Z) on the
slab's planes, and sum_x ||E_slab Z - d'||^2 = ||E Z - d||^2 (F_x is unitary). The Haar
transform of 8 x 8 tiles (J = 3) never crosses a slab boundary of whole tiles. What needs every
plane -- the Casorati Gram of step (1), the statistics, max |T(X_0)| -- goes through a record
laid out as the library's (sum part: data-consistency 4, sparse 2, zeros 2, the Gram 2 nz^2
as interleaved complex; max part: max |T(X_0)|), which the caller reduces over the slabs. The
singular-value thresholding uses the Gram route: G = V diag(sigma^2) V^H, W = V diag(sigma''/
sigma) V^H, L = (X - S) W (equal to U diag(sigma'') V^H, pinned in the oracle's tests).
"""
import numpy as np

from oracle import lps_oracle as O

HEAD = 8


class NumpySlab:
    def __init__(self, x0, nx, d_full, coils_full, mask, p, prior=None):
        import torch
        self.x0, self.nx, self.p = x0, nx, p
        self.coils = np.asarray(coils_full[:, :, x0:x0 + nx, :], np.complex128)
        self.mask = mask
        self.kz, self.ky = O.line_index(mask)
        self.nz, self.ny = self.coils.shape[1], self.coils.shape[3]
        self.nc = self.nz
        # hybrid samples of the slab's planes: orthonormal inverse DFT along kx
        self.dh = np.fft.ifft(np.asarray(d_full, np.complex128), axis=2, norm="ortho")[:, :, x0:x0 + nx]
        self.keep = None if prior is None else prior[0]
        self.sigma_prev = None if prior is None else prior[1]
        nn = self.nc * self.nc
        self.rec = torch.zeros(HEAD + 2 * nn + 1, dtype=torch.float64)
        self.nsum = HEAD + 2 * nn

    # ---- operators restricted to the slab (Sec. 2)
    def E(self, Z):
        out = np.empty((self.coils.shape[0], self.kz.size, self.nx), np.complex128)
        for c in range(self.coils.shape[0]):
            K = np.fft.fftn(self.coils[c] * Z, axes=(0, 2), norm="ortho")
            out[c] = K[self.kz, :, self.ky]
        return out

    def EH(self, R):
        X = np.zeros((self.nz, self.nx, self.ny), np.complex128)
        for c in range(self.coils.shape[0]):
            K = np.zeros_like(X)
            K[self.kz, :, self.ky] = R[c]
            X += np.conj(self.coils[c]) * np.fft.ifftn(K, axes=(0, 2), norm="ortho")
        return X

    def _put(self, gram, dc=(0.0, 0.0, 0.0), lrs=(0.0, 0.0), haar=None):
        r = self.rec.numpy()
        r[:HEAD] = 0.0
        r[0:3] = dc
        r[4:6] = lrs
        r[HEAD:self.nsum:2] = gram.real.ravel()
        r[HEAD + 1:self.nsum:2] = gram.imag.ravel()
        if haar is not None:
            r[self.nsum] = haar

    def _gram(self):
        r = self.rec.numpy()
        return (r[HEAD:self.nsum:2] + 1j * r[HEAD + 1:self.nsum:2]).reshape(self.nc, self.nc)

    # ---- Algorithm 1
    def begin(self):
        J = self.p.wavelet_levels
        self.X = self.EH(self.dh)                 # (0) X_0 = E^H d on the slab
        self.S = np.zeros_like(self.X)
        self.Lp = self.X.copy()                   # L_0 := X_0
        M = O.casorati(self.X)
        self._put(M.conj().T @ M, haar=float(np.max(np.abs(O.T(self.X, J)))))

    def iterate(self, k):
        p, J = self.p, self.p.wavelet_levels
        G = self._gram()
        lam, V = np.linalg.eigh(0.5 * (G + G.conj().T))
        order = np.argsort(lam)[::-1]
        lam, V = lam[order], V[:, order]
        s = np.sqrt(np.maximum(lam, 0.0))
        if k == 1:
            self.lamL = p.lambda_L_rel * s[0]
            self.lamS = p.lambda_S_rel * float(self.rec.numpy()[self.nsum])
        Z_old = self.Lp + self.S
        # (1)-(2): singular-value threshold, prior pull, rank guard, reprojection through W
        s1 = np.maximum(s - self.lamL, 0.0)
        s2 = s1 - p.lambda_p * (s1 - self.sigma_prev) if self.sigma_prev is not None else s1
        s2 = np.where(s <= p.rank_tau * s[0], 0.0, s2)
        f = np.where(s > 0, s2 / np.where(s > 0, s, 1.0), 0.0)
        W = (V * f) @ V.conj().T
        L = O.uncasorati(O.casorati(self.X - self.S) @ W, self.X.shape)
        # (3) sparsity off the prior support
        c = O.T(self.X - self.Lp, J)
        c2 = O.support_shrink(c, self.lamS, self.keep)
        S = O.Tinv(c2, J)
        # (4) data consistency
        R = self.E(L + S) - self.dh
        X = L + S - self.EH(R)
        self.X, self.S, self.Lp, self.c, self.sigma = X, S, L, c, s2
        Z = L + S
        off = np.ones(c.shape, bool) if self.keep is None else ~self.keep
        M = O.casorati(X - S)
        self._put(M.conj().T @ M,
                  dc=(float(np.vdot(R, R).real), float(np.vdot(Z - Z_old, Z - Z_old).real),
                      float(np.vdot(Z_old, Z_old).real)),
                  lrs=(float(np.abs(c2[off]).sum()), float((np.abs(c) > self.lamS).sum())))

    def end(self):
        return {"L": self.Lp, "S": self.S, "recon": self.Lp + self.S, "sigma": self.sigma,
                "support": np.abs(self.c) > self.lamS}
