"""Quadrature rules (oracle; test infrastructure only).

The paper computes the load vector by "high-order numerical integration"
(Section 4); the rules below are the oracle's choice: Gauss-Legendre nodes
found by Newton's method on the Legendre polynomial (three-term recurrence),
and a collapsed (Duffy) tensor rule on the reference triangle.
"""
from __future__ import annotations

import math
from functools import lru_cache

import numpy as np


def _legendre_and_derivative(n: int, x: np.ndarray):
    """P_n(x) and P_n'(x) by the recurrence (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1}."""
    p0 = np.ones_like(x)
    p1 = x.copy()
    if n == 0:
        return p0, np.zeros_like(x)
    for k in range(1, n):
        p0, p1 = p1, ((2 * k + 1) * x * p1 - k * p0) / (k + 1)
    # derivative: (1 - x^2) P_n' = n (P_{n-1} - x P_n)
    dp = n * (p0 - x * p1) / (1.0 - x * x)
    return p1, dp


@lru_cache(maxsize=None)
def gauss_legendre(n: int):
    """n-point Gauss-Legendre rule on [-1, 1] (exact for degree 2n-1)."""
    k = np.arange(1, n + 1, dtype=np.float64)
    x = np.cos(np.pi * (k - 0.25) / (n + 0.5))  # initial guesses
    for _ in range(100):
        p, dp = _legendre_and_derivative(n, x)
        dx = p / dp
        x = x - dx
        if np.max(np.abs(dx)) < 1e-16:
            break
    p, dp = _legendre_and_derivative(n, x)
    w = 2.0 / ((1.0 - x * x) * dp * dp)
    order = np.argsort(x)
    return x[order].copy(), w[order].copy()


def gauss_interval(n: int, a: float = 0.0, b: float = 1.0):
    """Gauss-Legendre rule mapped to [a, b]."""
    x, w = gauss_legendre(n)
    return 0.5 * (b - a) * x + 0.5 * (b + a), 0.5 * (b - a) * w


@lru_cache(maxsize=None)
def triangle_rule(n: int):
    """Collapsed Gauss rule on the reference triangle {xi, eta >= 0, xi + eta <= 1}.

    Maps the unit square (u, v) -> (xi, eta) = (u, v (1 - u)), Jacobian (1 - u);
    n x n points, exact for polynomials of total degree 2n - 2.
    Returns (xi, eta, w) with sum(w) = 1/2.
    """
    u, wu = gauss_interval(n, 0.0, 1.0)
    v, wv = gauss_interval(n, 0.0, 1.0)
    U, V = np.meshgrid(u, v, indexing="ij")
    WU, WV = np.meshgrid(wu, wv, indexing="ij")
    xi = U
    eta = V * (1.0 - U)
    w = WU * WV * (1.0 - U)
    return xi.ravel(), eta.ravel(), w.ravel()


def monomial_triangle_integral(a: int, b: int) -> float:
    """Exact integral of xi^a eta^b over the reference triangle: a! b! / (a + b + 2)!."""
    return math.factorial(a) * math.factorial(b) / math.factorial(a + b + 2)
