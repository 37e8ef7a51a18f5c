"""Seeded synthetic inputs shared by the oracle tests and the GPU parity tests.

This module only draws random numbers and moves them into place: it holds none
of the method's arithmetic (no transforms, products, projections or time
stepping), so that neither side of a parity test can inherit the other's
mistakes through it.

Layouts
  compact: ``a[f, kz+K, ky+K, kx]`` for |kz|, |ky| <= K and 0 <= kx <= K,
           K = (N-1)//3 by default -- the spectral state of the C ABI (fields
           u1, u2, u3, phi); another K (the cube holding a sphere) is given
           explicitly and read back from the array's last axis.
  full:    NumPy ``rfftn`` layout ``a[f, kz mod N, ky mod N, kx]`` with kx in [0, N/2].
"""
from __future__ import annotations

import numpy as np


def K_of(N: int) -> int:
    return (N - 1) // 3


def random_compact_state(N: int, seed: int, nfields: int = 4, kpeak: float = 4.0,
                         K: int | None = None, sphere: bool = False) -> np.ndarray:
    """Complex Gaussian modes with an envelope that peaks near |k| = kpeak and
    decays like a turbulent spectrum; kx = 0 plane made conjugate-symmetric
    (real fields), k = 0 set to zero.  Amplitudes are O(N^3) like the
    unnormalised DFT coefficients of an O(1) field.  ``sphere``: modes with
    9|k|^2 >= 2N^2 are zero (a state on the sphere |k| < sqrt(2) N/3)."""
    K = K_of(N) if K is None else K
    P, M = 2 * K + 1, K + 1
    rng = np.random.default_rng(seed)
    a = rng.standard_normal((nfields, P, P, M)) + 1j * rng.standard_normal((nfields, P, P, M))
    kz = np.arange(-K, K + 1).reshape(P, 1, 1)
    ky = np.arange(-K, K + 1).reshape(1, P, 1)
    kx = np.arange(0, M).reshape(1, 1, M)
    kk = np.sqrt(kx * kx + ky * ky + kz * kz) + 1e-30
    env = (kk / kpeak) ** 2 * np.exp(-(kk / kpeak) ** 2) / np.maximum(kk, 1.0)
    a = a * env[None] * float(N) ** 3 * 0.05
    if sphere:
        a = np.where((9 * (kx * kx + ky * ky + kz * kz) < 2 * N * N)[None], a, 0.0)
    # real fields: a(0, -ky, -kz) = conj(a(0, ky, kz))
    for iz in range(P):
        for iy in range(P):
            jz, jy = 2 * K - iz, 2 * K - iy
            if (iz, iy) > (jz, jy):
                a[:, iz, iy, 0] = np.conj(a[:, jz, jy, 0])
    a[:, K, K, 0] = 0.0
    return a


def compact_to_full(c: np.ndarray, N: int) -> np.ndarray:
    """Place a compact array into the zero-filled NumPy rfftn layout."""
    K = c.shape[-1] - 1
    nf = c.shape[0]
    out = np.zeros((nf, N, N, N // 2 + 1), dtype=np.complex128)
    idx = np.arange(-K, K + 1) % N
    out[:, idx[:, None], idx[None, :], : K + 1] = c
    return out


def full_to_compact(f: np.ndarray, N: int, K: int | None = None) -> np.ndarray:
    """Gather the modes |k_i| <= K of an rfftn-layout array into the compact layout."""
    K = K_of(N) if K is None else K
    idx = np.arange(-K, K + 1) % N
    return np.ascontiguousarray(f[:, idx[:, None], idx[None, :], : K + 1])
