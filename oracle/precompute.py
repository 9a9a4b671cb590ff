"""Row reduction and the closed-form local operators (FP64).

* Section IV-B: when A_s is not of full row rank, [A_s | b_s] is put in
  reduced row echelon form and the zero rows are dropped; a zero row whose
  right-hand side is not zero means the local system is inconsistent.
* Eq. (closed_2): with A_s of full row rank,
      Abar_s = A_s^T (A_s A_s^T)^{-1} A_s - I,
      bbar_s = A_s^T (A_s A_s^T)^{-1} b_s,
  and the local update is x_s = (1/rho) Abar_s d_s + bbar_s.

Readings (the paper gives no tolerance): a pivot is accepted when its
magnitude exceeds 1e-12 * max|A_s|; a reduced zero row is inconsistent when
|rhs| exceeds 1e-9 * max(1, max|b_s|).  Section III-B takes A_s of full row
rank and applies row reduction only when it is not: so the row reduction
always decides rank and consistency, and its rows replace A_s only for a
rank-deficient component.  (Reducing a full-rank block anyway can pivot on a
tiny impedance entry and leave a badly conditioned A_s A_s^T -- the
operators are the same in exact arithmetic, not in FP64.)
"""
from __future__ import annotations

import dataclasses

import numpy as np


class InconsistentError(ValueError):
    """Row reduction found 0 = b with b != 0 (library: OPF_ERR_INCONSISTENT)."""


def rref(A: np.ndarray, b: np.ndarray):
    """Reduced row echelon form of [A | b] by Gauss-Jordan elimination with
    partial pivoting; returns the nonzero rows (A_r, b_r) and the pivot
    columns.  Raises InconsistentError on a row 0 = b, b != 0."""
    A = np.array(A, dtype=np.float64, copy=True)
    b = np.array(b, dtype=np.float64, copy=True)
    m, n = A.shape
    if m == 0:
        return A, b, []
    tol = 1e-12 * max(np.abs(A).max(), 0.0)
    btol = 1e-9 * max(1.0, np.abs(b).max())
    M = np.hstack([A, b[:, None]])
    row = 0
    pivots = []
    for col in range(n):
        if row >= m:
            break
        r = row + int(np.argmax(np.abs(M[row:, col])))
        if abs(M[r, col]) <= tol:
            continue
        if r != row:
            M[[row, r]] = M[[r, row]]
        M[row] = M[row] / M[row, col]
        for k in range(m):
            if k != row and M[k, col] != 0.0:
                M[k] = M[k] - M[k, col] * M[row]
        pivots.append(col)
        row += 1
    for k in range(row, m):
        if abs(M[k, n]) > btol:
            raise InconsistentError(f"row reduction: 0 = {M[k, n]:.3e}")
    return M[:row, :n], M[:row, n], pivots


def closed_form(A: np.ndarray, b: np.ndarray):
    """Abar_s and bbar_s of Eq. (closed_2) for a full-row-rank A_s, with
    (A_s A_s^T)^{-1} applied through a Cholesky factorization."""
    m, n = A.shape
    if m == 0:
        return -np.eye(n), np.zeros(n)
    G = A @ A.T
    L = np.linalg.cholesky(G)
    # Y = G^{-1} A  (m x n), y = G^{-1} b
    Y = np.linalg.solve(L.T, np.linalg.solve(L, A))
    y = np.linalg.solve(L.T, np.linalg.solve(L, b))
    Abar = A.T @ Y - np.eye(n)
    bbar = A.T @ y
    return Abar, bbar


@dataclasses.dataclass
class Precomputed:
    Abar: list          # per component, n_s x n_s
    bbar: list          # per component, n_s
    Ared: list          # row-reduced A_s (full row rank)
    bred: list
    m_red: np.ndarray   # rows kept per component


def precompute(model) -> Precomputed:
    """Algorithm 1, precomputation: row reduction (when A_s is rank deficient)
    then Eq. (closed_2) per component."""
    Ab, bb, Ar, br, mr = [], [], [], [], []
    for comp in model.comps:
        A_r, b_r, _ = rref(comp.A, comp.b)
        if A_r.shape[0] == comp.A.shape[0]:      # already full row rank
            A_r, b_r = np.array(comp.A, dtype=np.float64), np.array(comp.b, dtype=np.float64)
        Abar, bbar = closed_form(A_r, b_r)
        Ab.append(Abar); bb.append(bbar); Ar.append(A_r); br.append(b_r)
        mr.append(A_r.shape[0])
    return Precomputed(Ab, bb, Ar, br, np.array(mr))
