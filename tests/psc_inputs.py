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


def separable_factors(N: int, seed: int, rank: int = 2, k0: float = 16.0, kc: float | None = None) -> list:
    """Random 1D spectral factors of a state whose fields are sums of products
    f(x) = sum_t a_t(x1) b_t(x2) c_t(x3): [u1 terms, u2 terms, u3 terms, phi terms],
    each term a triple (X, Y, Z) of complex arrays over k = -K..K (index k + K),
    K = (N-1)//3, conjugate-symmetric (real factors), zero at k = 0.

    The velocity is the curl of a random potential A whose components are sums
    of ``rank`` such products (u1 = d2 A3 - d3 A2, ...: i k applied to one
    factor), so it is solenoidal like the solver's states; phi is a sum of
    ``rank`` products.  Per-axis envelope exp(-|k|/kc) / (1 + (k/k0)^2)
    (kc = K/6 by default): a decaying spectrum that still leaves every
    retained wavenumber with content.  Coefficients are O(N^3) at
    their largest, like the unnormalised coefficients of an O(1) field."""
    K = K_of(N)
    kc = K / 6.0 if kc is None else kc
    k = np.arange(-K, K + 1)
    rng = np.random.default_rng(seed)
    env = np.exp(-np.abs(k) / kc) / (1.0 + (k / k0) ** 2)

    def draw(scale):
        terms = []
        for _ in range(rank):
            tri = []
            for _ in range(3):
                a = (rng.standard_normal(2 * K + 1) + 1j * rng.standard_normal(2 * K + 1)) * env * scale
                a[:K] = np.conj(a[K + 1:][::-1])  # a(-k) = conj(a(k))
                a[K] = 0.0
                tri.append(a)
            terms.append(tuple(tri))
        return terms

    A = [draw(1.0) for _ in range(3)]
    phi = draw(1.0)
    ik = 1j * k

    def d(terms, axis, sign=1.0):  # sign * d/dx_{axis+1}: i k on that factor, the sign on the first
        out = []
        for t in terms:
            t = [ik * a if i == axis else a for i, a in enumerate(t)]
            t[0] = sign * t[0]
            out.append(tuple(t))
        return out

    u1 = d(A[2], 1) + d(A[1], 2, -1.0)
    u2 = d(A[0], 2) + d(A[2], 0, -1.0)
    u3 = d(A[1], 0) + d(A[0], 1, -1.0)

    def normalise(fields):  # largest term coefficient 0.05 N^3
        top = max(np.abs(t[0]).max() * np.abs(t[1]).max() * np.abs(t[2]).max() for f in fields for t in f)
        c = 0.05 * float(N) ** 3 / top
        return [[(c * t[0], t[1], t[2]) for t in f] for f in fields]

    return normalise([u1, u2, u3]) + normalise([phi])


def separable_compact_state(factors: list, N: int, xp=np, dtype=None):
    """Materialise the compact state [f, kz+K, ky+K, kx] of separable factors:
    entry (kx, ky, kz) of field f is sum_t X_t(kx) Y_t(ky) Z_t(kz).  ``xp`` is
    numpy or torch (then ``dtype`` and a device come from the factors' tensors
    made by the caller)."""
    K = K_of(N)
    fields = []
    for terms in factors:
        acc = None
        for X, Y, Z in terms:
            t = Z[:, None, None] * Y[None, :, None] * X[None, None, K:]
            acc = t if acc is None else acc + t
        fields.append(acc)
    return xp.stack(fields)
