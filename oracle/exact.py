"""Exact PPR ground truth -- TEST INFRASTRUCTURE (see ``oracle/__init__.py``).

PPR of source s is the stopping distribution of the alpha-terminating walk
(Section 2.1).  In matrix form (Eq. (powerit), Section 6.3)

    pi_s = alpha * e_s + (1 - alpha) * pi_s P,   P = D^-1 A  (row-stochastic),

so pi_s solves (I - (1 - alpha) P^T) pi_s^T = alpha e_s.  ``dense_ppr`` solves
that system by LU (tiny graphs); ``power_iteration`` iterates the fixed point
(the ground truth of Section 8.3, "Power Iteration ... 100 iterations"), here
until the L1 change is below ``tol`` and at least ``min_iter`` times.
Edges count with multiplicity: a node with two parallel edges to u moves to u
with probability 2/d_out.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def transition_matrix(row_ptr, col):
    """Row-stochastic P = D^-1 A as a scipy CSR matrix (duplicates summed)."""
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    col = np.asarray(col, dtype=np.int64)
    n = len(row_ptr) - 1
    deg = np.diff(row_ptr)
    if np.any(deg == 0):
        raise ValueError("dangling node: every node needs d_out >= 1")
    rows = np.repeat(np.arange(n), deg)
    vals = 1.0 / deg[rows]
    return sp.csr_matrix((vals, (rows, col)), shape=(n, n))


def dense_ppr(row_ptr, col, alpha, sources):
    """Exact PPR rows pi(s, .) for each s by a dense LU solve; shape [len(sources), n]."""
    P = transition_matrix(row_ptr, col).toarray()
    n = P.shape[0]
    M = np.eye(n) - (1.0 - alpha) * P.T
    rhs = np.zeros((n, len(sources)))
    for i, s in enumerate(sources):
        rhs[s, i] = alpha
    return np.linalg.solve(M, rhs).T


def power_iteration(row_ptr, col, alpha, sources, tol=1e-15, min_iter=100, max_iter=2000):
    """PPR rows by iterating pi <- alpha e_s + (1 - alpha) pi P; shape [len(sources), n]."""
    PT = transition_matrix(row_ptr, col).T.tocsr()
    n = PT.shape[0]
    S = len(sources)
    E = np.zeros((n, S))
    E[np.asarray(sources), np.arange(S)] = alpha
    X = np.zeros((n, S))
    X[np.asarray(sources), np.arange(S)] = 1.0
    for it in range(max_iter):
        Xn = E + (1.0 - alpha) * (PT @ X)
        change = np.abs(Xn - X).sum(axis=0).max()
        X = Xn
        if it + 1 >= min_iter and change < tol:
            break
    return X.T
