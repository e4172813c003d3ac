"""FP64 oracle of the two-level (DD-alpha-AMG style) preconditioner.

TEST INFRASTRUCTURE ONLY (tests, smoke check, benchmark CPU legs). Plain
numpy over the oracle's own Wilson-clover operator (``oracle.Operator``).

The paper's method is DD-alpha-AMG (Sec. 1, reference [Frommer 2014]): an
aggregation-based coarse-grid correction whose fine-level smoother is the
Schwarz method of Sec. 3.1. The paper prints none of it; this is the
textbook two-level form of that method:

  * aggregates: lattice blocks; test vectors v_1..v_N (fine fields);
  * interpolation P: on every aggregate a and chirality h (spins {0,1} or
    {2,3}), the test vectors restricted to (a, h) orthonormalised by modified
    Gram-Schmidt in the order v_1, ..., v_N; coarse index (a, h, k);
  * coarse operator D_c = P^dagger D P (Galerkin);
  * preconditioner M r: e_c ~ D_c^-1 P^dagger r by GMRES(m_c) from zero on the
    coarse system, x = P e_c, then x += SAP(r - D x) (Schwarz post-smoothing);
  * outer FGMRES(m) right-preconditioned by M, true residual in FP64.

Nothing here builds the coarse operator's stencil: D_c is applied as
P^dagger (D (P c)), its definition.
"""
from __future__ import annotations

import numpy as np


def mgs_columns(W: np.ndarray) -> np.ndarray:
    """Modified Gram-Schmidt on the columns of W, in column order."""
    Q = np.array(W, dtype=np.complex128, copy=True)
    for k in range(Q.shape[1]):
        for j in range(k):
            Q[:, k] -= np.vdot(Q[:, j], Q[:, k]) * Q[:, j]
        Q[:, k] /= np.linalg.norm(Q[:, k])
    return Q


class TwoLevel:
    """Interpolation and coarse operator from given test vectors (N, V, 4, 3)."""

    def __init__(self, op, cblock, test_vectors):
        self.op = op
        self.cblock = tuple(cblock)
        tv = np.asarray(test_vectors, dtype=np.complex128).reshape(-1, op.V, 4, 3)
        self.N = tv.shape[0]
        self.nagg = op.nblocks(self.cblock)
        self.sites = [op.block_sites(self.cblock, a) for a in range(self.nagg)]
        # Q[a][h]: (|a| * 2 spins * 3 colours) x N, orthonormal columns
        self.Q = []
        for a in range(self.nagg):
            qa = []
            for h in range(2):
                W = tv[:, self.sites[a], 2 * h:2 * h + 2, :].reshape(self.N, -1).T
                qa.append(mgs_columns(W))
            self.Q.append(qa)

    # coarse vectors: (nagg, 2, N) complex
    def restrict(self, r) -> np.ndarray:
        r = np.asarray(r, dtype=np.complex128).reshape(self.op.V, 4, 3)
        c = np.empty((self.nagg, 2, self.N), dtype=np.complex128)
        for a in range(self.nagg):
            for h in range(2):
                c[a, h] = self.Q[a][h].conj().T @ r[self.sites[a], 2 * h:2 * h + 2, :].reshape(-1)
        return c

    def prolong(self, c) -> np.ndarray:
        c = np.asarray(c, dtype=np.complex128).reshape(self.nagg, 2, self.N)
        x = np.zeros((self.op.V, 4, 3), dtype=np.complex128)
        for a in range(self.nagg):
            for h in range(2):
                x[self.sites[a], 2 * h:2 * h + 2, :] = (self.Q[a][h] @ c[a, h]).reshape(-1, 2, 3)
        return x

    def coarse_apply(self, c) -> np.ndarray:
        """D_c c = P^dagger D P c."""
        return self.restrict(self.op.apply(self.prolong(c)))

    def coarse_gmres(self, rhs, restart: int, max_iter: int, tol: float) -> np.ndarray:
        """GMRES(restart) on D_c from zero, modified Gram-Schmidt, stopping when
        the estimated residual falls below tol * |rhs| or after max_iter steps."""
        b = np.asarray(rhs, dtype=np.complex128).reshape(-1)
        x = np.zeros_like(b)
        bn = np.linalg.norm(b)
        if bn == 0:
            return x.reshape(self.nagg, 2, self.N)
        its = 0
        r = b.copy()
        while its < max_iter:
            beta = np.linalg.norm(r)
            if beta <= tol * bn:
                break
            V = [r / beta]
            H = np.zeros((restart + 1, restart), dtype=np.complex128)
            k = 0
            for j in range(restart):
                w = self.coarse_apply(V[j]).reshape(-1)
                for i in range(j + 1):
                    H[i, j] = np.vdot(V[i], w)
                    w = w - H[i, j] * V[i]
                H[j + 1, j] = np.linalg.norm(w)
                its += 1
                k = j + 1
                e1 = np.zeros(k + 1, dtype=np.complex128)
                e1[0] = beta
                y, *_ = np.linalg.lstsq(H[:k + 1, :k], e1, rcond=None)
                est = np.linalg.norm(e1 - H[:k + 1, :k] @ y)
                if H[j + 1, j] == 0 or est <= tol * bn or its >= max_iter:
                    break
                V.append(w / H[j + 1, j])
            x = x + np.column_stack(V[:k]) @ y
            r = b - self.coarse_apply(x).reshape(-1)
            if est <= tol * bn:
                break
        return x.reshape(self.nagg, 2, self.N)

    def precondition(self, r, sap_block, sweeps: int, nmr: int, coarse_restart: int, coarse_iter: int,
                     coarse_tol: float) -> np.ndarray:
        """M r: coarse-grid correction, then Schwarz post-smoothing."""
        r = np.asarray(r, dtype=np.complex128).reshape(self.op.V, 4, 3)
        ec = self.coarse_gmres(self.restrict(r), coarse_restart, coarse_iter, coarse_tol)
        x = self.prolong(ec)
        return x + self.op.sap(sap_block, r - self.op.apply(x), sweeps, nmr)

    def fgmres(self, b, restart: int, tol: float, max_iter: int, **mkw):
        """FGMRES(restart) right-preconditioned by M. Returns (x, iterations)."""
        b = np.asarray(b, dtype=np.complex128).reshape(-1)
        bn = np.linalg.norm(b)
        x = np.zeros_like(b)
        its = 0
        while True:
            r = b - self.op.apply(x).reshape(-1)
            beta = np.linalg.norm(r)
            if beta <= tol * bn or its >= max_iter:
                return x.reshape(self.op.V, 4, 3), its
            V, Z = [r / beta], []
            H = np.zeros((restart + 1, restart), dtype=np.complex128)
            k = 0
            for j in range(restart):
                z = self.precondition(V[j], **mkw).reshape(-1)
                Z.append(z)
                w = self.op.apply(z).reshape(-1)
                for i in range(j + 1):
                    H[i, j] = np.vdot(V[i], w)
                    w = w - H[i, j] * V[i]
                H[j + 1, j] = np.linalg.norm(w)
                its += 1
                k = j + 1
                e1 = np.zeros(k + 1, dtype=np.complex128)
                e1[0] = beta
                y, *_ = np.linalg.lstsq(H[:k + 1, :k], e1, rcond=None)
                est = np.linalg.norm(e1 - H[:k + 1, :k] @ y)
                if H[j + 1, j] == 0 or est <= tol * bn or its >= max_iter:
                    break
                V.append(w / H[j + 1, j])
            x = x + np.column_stack(Z[:k]) @ y
