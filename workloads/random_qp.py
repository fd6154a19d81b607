"""Seeded random dense QPs with equality and inequality rows: the stand-in for
the random-QP benchmark of Sec. V-A (ten sizes n log-spaced from 10 to 2000,
n/4 equality and n/4 inequality constraints, ten problems per size, solved
to residuals below 1e-6).

The paper does not print its generator; this one (a reading) draws

    P = M M^T / n + 0.01 I          (M ~ N(0, 1), n x n: SPD, condition ~ 400)
    q ~ N(0, 1)
    A ~ N(0, 1) / sqrt(n)           ((n/4 + n/4) x n, so that |A x| ~ |x|)
    x_f ~ N(0, 1)                   (a feasible point)
    rows [0, n/4):      l = u = A x_f              (equalities)
    rows [n/4, n/2):    l = -inf, u = A x_f + U[0, 1]   (one-sided inequalities)

so that the problem is feasible by construction and a part of the
inequalities binds at the optimum.  Like ``workloads.mpc`` it only builds
problems: none of the solver's arithmetic is here.
"""
from __future__ import annotations

import numpy as np

from .mpc import rng_for

WORKLOAD_ID = 91

# ten sizes logarithmically spaced from 10 to 2000 (rounded)
SIZES = tuple(int(round(v)) for v in np.logspace(1.0, np.log10(2000.0), 10))


def random_dense_qp(seed: int, n: int):
    """(P, q, A, l, u) of random problem `seed` of size n (n/4 equality rows first)."""
    rng = rng_for(WORKLOAD_ID, seed * 100000 + n)
    me = n // 4
    mi = n // 4
    M = rng.standard_normal((n, n))
    P = M @ M.T / n + 1e-2 * np.eye(n)
    P = 0.5 * (P + P.T)
    q = rng.standard_normal(n)
    A = rng.standard_normal((me + mi, n)) / np.sqrt(n)
    xf = rng.standard_normal(n)
    Ax = A @ xf
    l = np.empty(me + mi)
    u = np.empty(me + mi)
    l[:me] = Ax[:me]
    u[:me] = Ax[:me]
    l[me:] = -np.inf
    u[me:] = Ax[me:] + rng.uniform(0.0, 1.0, mi)
    return P, q, A, l, u
