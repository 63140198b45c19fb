"""Banded Cholesky and Takahashi selected inversion (Sec. 3.2).

Test infrastructure (see the package docstring).  Natural (lexicographic,
time-major) ordering: for the structured-grid stencils the Cholesky factor
fills exactly the band, so no reordering is needed.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp


def bandwidth(Q: sp.spmatrix) -> int:
    C = Q.tocoo()
    return int(np.max(np.abs(C.row - C.col))) if C.nnz else 0


def to_lower_band(Q: sp.spmatrix, bw: int | None = None) -> np.ndarray:
    """LAPACK lower band storage ab[i - j, j] = Q[i, j], i >= j."""
    Q = Q.tocsr()
    N = Q.shape[0]
    if bw is None:
        bw = bandwidth(Q)
    ab = np.zeros((bw + 1, N))
    C = Q.tocoo()
    offs = np.unique(C.row - C.col)
    for d in offs[offs >= 0]:
        ab[d, : N - d] = Q.diagonal(-int(d))
    return ab


def cholesky(Q: sp.spmatrix) -> np.ndarray:
    """Lower banded Cholesky factor, Q = L L^T (LAPACK pbtrf); raises
    numpy.linalg.LinAlgError if Q is not positive definite."""
    return sla.cholesky_banded(to_lower_band(Q), lower=True)


def solve(Lb: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Q^-1 b from the banded factor: one forward and one backward solve."""
    return sla.cho_solve_banded((Lb, True), b)


def backward_solve(Lb: np.ndarray, z: np.ndarray) -> np.ndarray:
    """L^-T z (Cholesky sampling: mu + L^-T z ~ N(mu, Q^-1), Sec. 3.2)."""
    bw = Lb.shape[0] - 1
    N = Lb.shape[1]
    # L^T is upper banded with ab_up[bw + i - j, j] = L^T[i, j] = L[j, i]
    ab_up = np.zeros_like(Lb)
    for d in range(bw + 1):
        ab_up[bw - d, d:] = Lb[d, : N - d]
    return sla.solve_banded((0, bw), ab_up, z)


def logdet(Lb: np.ndarray) -> float:
    return 2.0 * float(np.sum(np.log(Lb[0])))


def takahashi_diag(Lb: np.ndarray) -> np.ndarray:
    """diag(Q^-1) by the Takahashi recursion on the band (Rue & Martino
    2007; Sec. 3.2 "Marginal variance computation"):
    Sigma_ij = delta_ij / L_ii^2 - (1/L_ii) sum_{k>i} L_ki Sigma_kj, j >= i,
    run for i = N-1 .. 0 over a sliding dense window of the band."""
    bw = Lb.shape[0] - 1
    N = Lb.shape[1]
    win = np.zeros((bw + 1, bw + 1))        # win[a, b] = Sigma[i + a, i + b]
    out = np.empty(N)
    for i in range(N - 1, -1, -1):
        w = min(bw, N - 1 - i)
        new = np.zeros_like(win)
        new[1:, 1:] = win[:bw, :bw]
        lii = Lb[0, i]
        l = Lb[1: w + 1, i]                    # L[i+1 .. i+w, i]
        W = new[1: w + 1, 1: w + 1]
        s = -(l @ W) / lii                     # Sigma[i, i+1 .. i+w]
        new[0, 1: w + 1] = s
        new[1: w + 1, 0] = s
        new[0, 0] = 1.0 / lii ** 2 - (l @ s) / lii
        win = new
        out[i] = new[0, 0]
    return out
