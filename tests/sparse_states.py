"""Full-size right-hand-side checks on sparse states: the CUDA path against the
oracle's triad-by-triad sums (oracle.rhs_sparse_triads), for grids the oracle
cannot transform in a test.  Used by the GPU tests only."""
import numpy as np

from oracle import psc_oracle as O


def sparse_modes(N, seed, K, sphere):
    """Twelve modes from low k to the edge of the retained set (the 2/3 cube of
    half-width K, or the sphere 9|k|^2 < 2N^2 inside the cube of half-width K),
    with conjugate partners on kx = 0; amplitudes O(N^3)."""
    rng = np.random.default_rng(seed)
    if sphere:
        K = O.sphere_halfwidth(N)  # the sphere's edge (the stored cube may be one plane wider)
        e = int(K / np.sqrt(2.0))  # |(e, e, 0)| stays inside the sphere
        ks = [(1, 0, 1), (0, 2, -1), (2, 1, 0), (1, -1, 2), (3, 2, -2), (K, 0, 1), (0, K - 1, 2),
              (e, -e, 0), (e - 3, 2, e), (0, 1, 1), (K // 3, K // 2, -K // 2), (2, 0, 0)]
    else:
        ks = [(1, 0, 1), (0, 2, -1), (2, 1, 0), (1, -1, 2), (3, 2, -2), (5, -4, 1), (K, -K, 7),
              (K - 3, K, -K), (K * 3 // 5, -K * 4 // 9, K // 4), (0, 1, 1), (K // 3, K, 0), (2, 0, 0)]
    modes = {}
    for k in ks:
        if sphere:
            assert 9 * (k[0] ** 2 + k[1] ** 2 + k[2] ** 2) < 2 * N * N
        assert max(abs(c) for c in k) <= K
        v = (rng.standard_normal(4) + 1j * rng.standard_normal(4)) * float(N) ** 3 * 0.05
        modes[k] = v
        if k[0] == 0:
            modes[(0, -k[1], -k[2])] = np.conj(v)
    return modes


def check_sparse_rhs(torch, B, sim, seed):
    """One right-hand side of a sparse state through `sim` (a binding
    Simulation) against the triad sums: relative L2 and per-mode error within
    the one-RHS tolerance (2e-6 FP32-mixed, 1e-13 FP64), every other mode only
    round-off spread by the transforms (< 5x that tolerance of the largest)."""
    p = sim.p
    N, dl, prec = p.N, p.dealias, p.precision
    K = B.retained_halfwidth(N, dl)
    modes = sparse_modes(N, seed, K, dl == B.DEALIAS_PHASE_SHIFT)
    dev = sim.device
    cdt = torch.complex64 if prec == B.FP32_MIXED else torch.complex128
    x = torch.zeros(B.compact_shape(N, dl), dtype=cdt, device=dev)
    rounded = {}
    for (kx, ky, kz), v in modes.items():
        vv = v.astype(np.complex64) if prec == B.FP32_MIXED else v
        rounded[(kx, ky, kz)] = vv.astype(np.complex128)
        x[:, kz + K, ky + K, kx] = torch.from_numpy(vv).to(dev)
    out = sim.rhs(x)
    ref = O.rhs_sparse_triads(rounded, N, O.Params(N=N, nu=p.nu, Sc=p.Sc, beta=p.beta, eps_inj=p.eps_inj,
                                                   kF=p.kF, forcing=p.forcing, scalar_on=p.scalar_on,
                                                   dealias=dl))
    scale = max(np.abs(v).max() for v in ref.values())
    mask = torch.zeros(B.compact_shape(N, dl)[1:], dtype=torch.bool, device=dev)
    got, want = [], []
    for (kx, ky, kz), v in ref.items():
        got.append(out[:, kz + K, ky + K, kx].cpu().numpy().astype(np.complex128))
        want.append(v)
        mask[kz + K, ky + K, kx] = True
    got, want = np.array(got), np.array(want)
    tol = 2e-6 if prec == B.FP32_MIXED else 1e-13
    assert np.linalg.norm(got - want) / np.linalg.norm(want) < tol
    assert np.abs(got - want).max() < tol * scale
    # every other mode holds only round-off spread by the transforms: no single
    # element's error may exceed tol times the norm of the exact output (an
    # element's error is at most the L2 error of the whole output; the L2 sum
    # over the ~10^9 zero modes of a sparse state is the dense tests' concern)
    out[:, mask] = 0
    rest = float(out.abs().max())
    assert rest < tol * np.linalg.norm(want), (rest / np.linalg.norm(want), rest / scale)
