"""Nonnegative completion of one slice by the alternating direction method (App. A),
in float64 with the dense Z of the appendix (test infrastructure only).

The problem: minimise ||P_Omega(X Y - M)||_F^2 with X (m' x q), Y (q x n') >= 0,
rewritten with Z (equal to M on Omega), X = U, Y = V, U, V >= 0 and multipliers
Lambda (m' x q), Pi (q x n'); one iteration of App. A updates, in this order:

    X <- (Z Y^T + alpha U - Lambda) (Y Y^T + alpha I)^-1
    Y <- (X^T X + beta I)^-1 (X^T Z + beta V - Pi)
    Z <- X Y + P_Omega(M - X Y)
    U <- max(0, X + Lambda / alpha),  V <- max(0, Y + Pi / beta)
    Lambda <- Lambda + gamma alpha (X - U),  Pi <- Pi + gamma beta (Y - V)

Readings of the appendix where the printed text cannot hold: the Y step uses
X^T Z (the printed X Z^T has the wrong shape); the Lambda step adds to Lambda_k
(the printed right-hand side repeats Lambda_{k+1}); P_Omega keeps the entries in
Omega and zeros the others (so that Z equals M on Omega, which the Z step needs);
"X, Y > 0" is read as >= 0.  Parameters the paper does not give: alpha =
alpha_rel ||Y0||_F^2 / q and beta = alpha_rel ||X0||_F^2 / q (the mean Gram diagonal
of the start, as the ALS ridge term; alpha_rel 0.3), constant over the iterations,
and gamma = 1 (inside the stated interval (0, 1.618)).  Start: Y0^T[j][k] = sqrt(mu / q) (0.5 + w / 2^32) with
w from Philox (k, j, slice, 3) (the ALS start) and X0[i][k] likewise from Philox
(k, i, slice, 6); U0 = X0, V0 = Y0, Lambda0 = Pi0 = 0, Z0 = X0 Y0 + P_Omega(M - X0 Y0).
A fixed number of iterations is run (the paper stops on a tolerance or at 100).
"""
from __future__ import annotations

import numpy as np

from . import philox
from .als import init_v

TAG_ADM_X0 = 6


def init_x(seed: int, s: int, m_s: int, r: int, mu: float) -> np.ndarray:
    k = np.arange(r, dtype=np.uint64)[None, :]
    i = np.arange(m_s, dtype=np.uint64)[:, None]
    w = philox.draw(seed, k, i, s, TAG_ADM_X0)[0].astype(np.float64)
    return np.sqrt(max(mu, 0.0) / r) * (0.5 + w / 2.0 ** 32)


def penalty(F, alpha_rel: float) -> float:
    """alpha_rel times the mean diagonal of the Gram F^T F of a start factor F [n, q]."""
    F = np.asarray(F, dtype=np.float64)
    return alpha_rel * float(np.sum(F * F)) / max(F.shape[1], 1)


def complete_slice_adm(rows, cols, vals, m_s: int, n_s: int, r: int, iters: int, alpha_rel: float, gamma: float,
                       seed: int, s: int, X0=None, Y0=None, history=None, state=None):
    """Returns (X [m', q], Y^T [n', q]) after `iters` iterations.  X0 [m', q] and
    Y0 [n', q] (Y transposed) replace the seeded start; `history`, a list, receives
    ||P_Omega(X Y - M)||_F after every iteration; `state`, a dict, receives the
    final U, V^T, Lambda and Pi^T."""
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    vals = np.asarray(vals, dtype=np.float64)
    mu = float(vals.mean()) if vals.size else 0.0
    X = init_x(seed, s, m_s, r, mu) if X0 is None else np.array(X0, dtype=np.float64)
    Y = (init_v(seed, s, n_s, r, mu) if Y0 is None else np.array(Y0, dtype=np.float64)).T.copy()
    if vals.size == 0 or mu <= 0.0:
        # nothing observed, or an all-zero (nonnegative) slice: the zero factors fit
        return np.zeros((m_s, r)), np.zeros((n_s, r))
    mask = np.zeros((m_s, n_s), dtype=bool)
    mask[rows, cols] = True
    M = np.zeros((m_s, n_s))
    M[rows, cols] = vals
    alpha = penalty(Y.T, alpha_rel)
    beta = penalty(X, alpha_rel)
    I = np.eye(r)
    U, V = X.copy(), Y.copy()
    Lam, Pi = np.zeros_like(X), np.zeros_like(Y)
    XY = X @ Y
    Z = np.where(mask, M, XY)
    for _ in range(iters):
        X = (Z @ Y.T + alpha * U - Lam) @ np.linalg.inv(Y @ Y.T + alpha * I)
        Y = np.linalg.inv(X.T @ X + beta * I) @ (X.T @ Z + beta * V - Pi)
        XY = X @ Y
        Z = np.where(mask, M, XY)
        U = np.maximum(0.0, X + Lam / alpha)
        V = np.maximum(0.0, Y + Pi / beta)
        Lam = Lam + gamma * alpha * (X - U)
        Pi = Pi + gamma * beta * (Y - V)
        if history is not None:
            history.append(float(np.linalg.norm((XY - M)[mask])))
    if state is not None:
        state.update(U=U, VT=V.T, Lam=Lam, PiT=Pi.T)
    return X, Y.T
