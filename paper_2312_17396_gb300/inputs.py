"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds no arithmetic of the method: it only draws matrices (numpy
``default_rng``) and rescales them to a requested 1-norm.  Both the CUDA path and the
CPU oracle are fed from here by the tests and the benchmark.
"""
from __future__ import annotations

import numpy as np


# Rescaled matrices land a relative 2^-40 below the requested 1-norm, so that a target
# that is a power of two (||A||_1 = 4, 32) is not pushed across the boundary of the
# squaring count ceil(log2 ||A||_1) by the rounding of one summation order or another.
_BELOW = 1.0 - 2.0 ** -40


def gaussian_matrix(n: int, seed: int, norm1: float | None = None, scale: float = 1.0):
    """N(0,1) entries (times scale), optionally rescaled so that ||A||_1 = norm1."""
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, n)) * scale
    if norm1 is not None:
        A *= norm1 * _BELOW / np.abs(A).sum(axis=0).max()
    return A


def gaussian_batch(batch: int, n: int, seed: int, norm1=None, scale: float = 1.0):
    """batch x n x n N(0,1) matrices; norm1 a scalar or per-matrix array of 1-norms."""
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((batch, n, n)) * scale
    if norm1 is not None:
        target = np.broadcast_to(np.asarray(norm1, dtype=np.float64), (batch,))
        cur = np.abs(A).sum(axis=1).max(axis=1)
        A *= (target * _BELOW / cur)[:, None, None]
    return A


def uneven_batch(count: int, n_lo: int, n_hi: int, norm_lo: float, norm_hi: float, seed: int,
                 degrees=(12, 18, 24)):
    """Uneven batch: n uniform in [n_lo, n_hi], ||A||_1 log-uniform in [norm_lo, norm_hi],
    degree drawn uniformly from `degrees`.  Returns (list of matrices, list of degrees)."""
    rng = np.random.default_rng(seed)
    ns = rng.integers(n_lo, n_hi + 1, size=count)
    norms = np.exp(rng.uniform(np.log(norm_lo), np.log(norm_hi), size=count))
    degs = rng.choice(np.asarray(degrees), size=count)
    mats = []
    for k in range(count):
        A = rng.standard_normal((ns[k], ns[k]))
        A *= norms[k] * _BELOW / np.abs(A).sum(axis=0).max()
        mats.append(A)
    return mats, [int(d) for d in degs]


def prescribed_eigen_matrix(n: int, seed: int, lo: float = -8.0, hi: float = 8.0):
    """Q diag(lambda) Q^T with Q Haar-orthogonal (QR of a Gaussian, signs fixed) and
    lambda uniform in [lo, hi]."""
    rng = np.random.default_rng(seed)
    Z = rng.standard_normal((n, n))
    Q, R = np.linalg.qr(Z)
    Q *= np.sign(np.diag(R))[None, :]
    lam = rng.uniform(lo, hi, size=n)
    return (Q * lam[None, :]) @ Q.T


def strictly_upper(n: int, seed: int, scale: float = 100.0):
    """scale * triu(randn(n), 1): nilpotent (Section 3.4.3 class B)."""
    rng = np.random.default_rng(seed)
    return scale * np.triu(rng.standard_normal((n, n)), 1)
