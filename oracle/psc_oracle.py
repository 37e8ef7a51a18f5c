"""Plain FP64 CPU oracle for the pseudo-spectral forced-HIT + passive-scalar time step.

TEST INFRASTRUCTURE ONLY.  This module is imported by ``tests/``, by
``__graft_entry__.smoke()`` and by the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py``.  The product path (the CUDA library and its Python
binding) never imports, links or executes anything here, and this module
shares no code with it.

Everything is written straight from the paper's statement of the method
(arXiv:2012.04838, section 2), in float64/complex128 NumPy, with NumPy's FFT as
the only library primitive.  Arrays keep NumPy's ``rfftn`` layout: a physical
field is ``a[z, y, x]`` with ``x_j = 2*pi*j/N`` and its transform is
``ah[kz, ky, kx]`` with ``kx in [0, N/2]`` and ``ky, kz`` in FFT order.
Velocity arrays carry the component first: ``uh[c]`` with c = 0, 1, 2 for the
x1, x2, x3 directions.

Readings of the paper that the oracle adopts (the GPU path adopts the same):
  * 2/3-rule truncation: keep ``|k_i| <= K = floor((N-1)/3)`` on every axis.
  * rotational nonlinear term ``P(u x omega)`` (equal to ``-P(u.grad u)`` on
    the retained set; both forms are implemented, selectable by
    ``nonlinear_form``, and their agreement is a test).
  * constant-power forcing ``A = eps_inj / (2 E_f)`` on the sphere
    ``0 < |k|^2 <= k_F^2``, evaluated at every stage input; or the paper's
    deterministic variant (section 2.3), applied after the last stage: the
    band is rescaled so that its energy stays at its value at the first step.
  * Lawson integrating-factor RK4 for the viscous/diffusive terms; plain
    explicit RK4 (section 2.2) as the alternative integrator.
  * shells ``n = floor(|k| + 1/2)``; ``E(n) = sum w_k |u_k|^2 / (2 N^6)``.

Parity: every function below is pinned by ``tests/test_oracle_pins.py``
except where its docstring says "parity unpinned".
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# --------------------------------------------------------------------------
# Parameters (Table 2 of the paper plus the scalar inputs of section 2.3)
# --------------------------------------------------------------------------

FORCE_NONE = 0
FORCE_CONST_POWER = 1
FORCE_HOLD_ENERGY = 2       # the paper's deterministic scheme: band energy held after each step

IC_SPECTRUM_K4 = 0          # E(k) ~ k^4 exp(-2 (k/4)^2), random phases
IC_TAYLOR_GREEN_NOISE = 1   # Taylor-Green vortex plus the k^4 noise
IC_PAPER_EQ9 = 2            # Eq. 9 shape (k/kF)^2 below kF, (k/kF)^(-5/3) above

INTEG_IFRK4 = 0
INTEG_RK4 = 1

NL_ROTATIONAL = 0           # P(u x omega)
NL_CONVECTIVE = 1           # -P((u.grad) u), the form the paper writes (section 2.3)

DEALIAS_TWO_THIRDS = 0      # keep |k_i| <= (N-1)//3
DEALIAS_PHASE_SHIFT = 1     # the paper's: keep |k| < sqrt(2) N / 3, phase-shifted products


@dataclasses.dataclass
class Params:
    """Problem statement: grid N on [0, 2pi]^3, viscosity nu, Schmidt number Sc,
    mean scalar gradient beta along x2 (Eq. 3), forcing band kF and power eps_inj
    (section 2.3), time step dt (or CFL target, Eq. 10), IC seed and energy."""
    N: int = 32
    nu: float = 0.02
    Sc: float = 1.0
    beta: float = 1.0
    forcing: int = FORCE_CONST_POWER
    kF: float = 2.0
    eps_inj: float = 0.1
    dt: float = 0.005
    cfl: float = 0.0
    seed: int = 1
    ic: int = IC_TAYLOR_GREEN_NOISE
    ic_energy: float = 1.5
    ic_noise_frac: float = 0.01
    integrator: int = INTEG_IFRK4
    scalar_on: int = 1
    record_every: int = 10
    nonlinear_form: int = NL_ROTATIONAL
    dealias: int = DEALIAS_TWO_THIRDS

    @property
    def D(self) -> float:
        """Scalar diffusivity D = nu / Sc (section 2.3)."""
        return self.nu / self.Sc


# --------------------------------------------------------------------------
# Grid, wavenumbers and the DFT convention (Eqs. 4-5)
# --------------------------------------------------------------------------

def sphere_halfwidth(N: int) -> int:
    """Largest integer k with k < sqrt(2) N / 3, i.e. 9 k^2 < 2 N^2."""
    k = 0
    while 9 * (k + 1) ** 2 < 2 * N * N:
        k += 1
    return k


class Grid:
    """Periodic box of side 2*pi with N^3 points (Eq. 4) and its wavenumbers.

    ``kx, ky, kz`` are integer wavenumbers broadcastable against an
    ``rfftn`` array; ``k2 = |k|^2``; ``mask`` is the retained set: the 2/3-rule
    cube |k_i| <= K = (N-1)//3, or (``dealias`` = DEALIAS_PHASE_SHIFT) the
    paper's sphere |k| < sqrt(2) N / 3 (section 2.3), whose products are then
    formed on the grid and on the grid shifted by half a cell (``shifts``);
    ``w`` counts each stored mode together with its conjugate partner (1 on
    the kx = 0 plane, 2 elsewhere)."""

    def __init__(self, N: int, dealias: int = DEALIAS_TWO_THIRDS):
        if N < 8:
            raise ValueError("N must be at least 8")
        self.N = N
        self.dealias = dealias
        kfull = np.fft.fftfreq(N, 1.0 / N).round().astype(np.int64)
        self.kz = kfull.reshape(N, 1, 1)
        self.ky = kfull.reshape(1, N, 1)
        self.kx = np.arange(N // 2 + 1, dtype=np.int64).reshape(1, 1, N // 2 + 1)
        self.k2 = self.kx ** 2 + self.ky ** 2 + self.kz ** 2
        if dealias == DEALIAS_PHASE_SHIFT:
            self.K = sphere_halfwidth(N)
            self.mask = 9 * self.k2 < 2 * N * N
            self.shifts = (0, 1)
        else:
            self.K = (N - 1) // 3
            K = self.K
            self.mask = ((np.abs(self.kx) <= K) & (np.abs(self.ky) <= K)
                         & (np.abs(self.kz) <= K))
            self.shifts = (0,)
        self.w = np.where(self.kx == 0, 1.0, 2.0) * np.ones((N, N, 1))
        self.dx = 2.0 * np.pi / N
        c = self.dx * np.arange(N)
        self.z = c.reshape(N, 1, 1)
        self.y = c.reshape(1, N, 1)
        self.x = c.reshape(1, 1, N)

    @property
    def kvec(self):
        return (self.kx, self.ky, self.kz)

    def phase(self, shift: int):
        """exp(i k.delta) with delta = shift * (pi/N)(1, 1, 1): a field sampled
        at x + delta has the coefficients phase * u_hat (Patterson and Orszag
        1971).  Averaging a product formed at shifts 0 and 1 cancels every
        alias wrapped an odd number of times; the sphere removes the rest."""
        return np.exp(1j * shift * (np.pi / self.N) * (self.kx + self.ky + self.kz))

    @property
    def shape_hat(self):
        return (self.N, self.N, self.N // 2 + 1)


def fwd(a: np.ndarray) -> np.ndarray:
    """Forward DFT of Eq. 5: phi_hat_k = sum_x phi(x) exp(-i k.x), unnormalised."""
    return np.fft.rfftn(a)


def inv(ah: np.ndarray, N: int) -> np.ndarray:
    """Inverse DFT of Eq. 5: phi(x) = N^-3 sum_k phi_hat_k exp(i k.x)."""
    return np.fft.irfftn(ah, s=(N, N, N), axes=(0, 1, 2))


def truncate(ah: np.ndarray, g: Grid) -> np.ndarray:
    """Dealiasing: zero every mode outside the retained set (section 2.3)."""
    return np.where(g.mask, ah, 0.0)


def dealiased_products(fields_hat, product, g: Grid):
    """The transforms of product(*physical fields) on the retained set, the
    fields given by their transforms: one evaluation on the grid (2/3 rule), or
    the average of the evaluations on the grid and on the half-cell-shifted
    grid (phase-shift dealiasing).  product returns a list of physical fields."""
    acc = None
    for s in g.shifts:
        ph = g.phase(s)
        phys = [inv(ph * fh, g.N) for fh in fields_hat]
        outs = [np.conj(ph) * fwd(o) for o in product(*phys)]
        acc = outs if acc is None else [a + b for a, b in zip(acc, outs)]
    return [truncate(a / len(g.shifts), g) for a in acc]


# --------------------------------------------------------------------------
# Spectral operators (Eqs. 6-8)
# --------------------------------------------------------------------------

def grad_hat(ah: np.ndarray, g: Grid):
    """i k phi_hat: the transform of grad phi."""
    return [1j * kc * ah for kc in g.kvec]


def curl_hat(uh, g: Grid):
    """i k x u_hat: the transform of the vorticity omega = curl u."""
    kx, ky, kz = g.kvec
    return [1j * (ky * uh[2] - kz * uh[1]),
            1j * (kz * uh[0] - kx * uh[2]),
            1j * (kx * uh[1] - ky * uh[0])]


def project(fh, g: Grid):
    """Leray projection of Eq. 7: f - k (k.f)/|k|^2, which removes the
    pressure gradient (p_hat = i k.(u.grad u)_hat / |k|^2).  k = 0 maps to 0."""
    kdotf = sum(kc * fc for kc, fc in zip(g.kvec, fh))
    k2 = np.where(g.k2 == 0, 1, g.k2)
    out = [fc - kc * kdotf / k2 for kc, fc in zip(g.kvec, fh)]
    return [np.where(g.k2 == 0, 0.0, o) for o in out]


def velocity(uh, g: Grid):
    return [inv(uh[c], g.N) for c in range(3)]


def nonlinear_rotational(uh, g: Grid):
    """Projected, dealiased rotational nonlinear term P[(u x omega)_hat] on R.

    The NS right-hand side of Eq. 7 without the viscous and forcing terms:
    -u.grad u = u x omega - grad(|u|^2/2), and the gradient is removed by P."""
    def cross(u1, u2, u3, w1, w2, w3):
        return [u2 * w3 - u3 * w2, u3 * w1 - u1 * w3, u1 * w2 - u2 * w1]
    return project(dealiased_products(list(uh) + list(curl_hat(uh, g)), cross, g), g)


def nonlinear_convective(uh, g: Grid):
    """-P[(u.grad u)_hat] on R, the form the paper writes in Eqs. 6-7
    (velocity and its gradient transformed back separately, section 2.3)."""
    grads = [c for i in range(3) for c in grad_hat(uh[i], g)]  # d_j u_i at 3 i + j

    def adv(u1, u2, u3, *d):
        return [-(u1 * d[3 * i] + u2 * d[3 * i + 1] + u3 * d[3 * i + 2]) for i in range(3)]
    return project(dealiased_products(list(uh) + grads, adv, g), g)


def pressure_hat(uh, g: Grid):
    """The modified pressure of section 2.2 on R: taking the divergence of the
    momentum equation gives p_hat = i k.(u.grad u)_hat / |k|^2 (Eq. 6), with
    the convective term formed as the paper forms it (u and i k u_hat
    transformed back separately) and truncated to R; the forcing term drops
    out because A u is solenoidal.  p_hat = 0 at k = 0."""
    u = velocity(uh, g)
    adv = []
    for i in range(3):
        gi = [inv(c, g.N) for c in grad_hat(uh[i], g)]
        adv.append(truncate(fwd(u[0] * gi[0] + u[1] * gi[1] + u[2] * gi[2]), g))
    kdot = sum(kc * a for kc, a in zip(g.kvec, adv))
    k2 = np.where(g.k2 == 0, 1, g.k2)
    return np.where(g.k2 == 0, 0.0, 1j * kdot / k2)


def scalar_advection(uh, ph, g: Grid):
    """(u.grad phi)_hat on R (Eq. 8), formed in physical space from the
    inverse transforms of u_hat and i k phi_hat."""
    def dot(u1, u2, u3, g1, g2, g3):
        return [u1 * g1 + u2 * g2 + u3 * g3]
    return dealiased_products(list(uh) + list(grad_hat(ph, g)), dot, g)[0]


# --------------------------------------------------------------------------
# Forcing (section 2.3: energy injected on the sphere 0 < |k| <= kF)
# --------------------------------------------------------------------------

def band(g: Grid, kF: float) -> np.ndarray:
    return (g.k2 > 0) & (g.k2 <= kF * kF) & g.mask


def forced_energy(uh, g: Grid, kF: float) -> float:
    """E_f = sum over the forced sphere of w |u_hat|^2 / (2 N^6)."""
    b = band(g, kF)
    e = sum((np.abs(uh[c]) ** 2) for c in range(3))
    return float(np.sum(np.where(b, g.w * e, 0.0)) / (2.0 * g.N ** 6))


def hold_band_energy(uh, g: Grid, kF: float, Ef0: float):
    """The deterministic forcing of section 2.3, applied after the last RK
    stage: the modes of the sphere 0 < |k| <= kF are multiplied by
    f = sqrt(Ef0 / E_f) so that the band energy returns to Ef0 (E_f the band
    energy after the step; f = 1 if the band is empty).  Multiplying by f over
    a step of length dt is forcing with the rate A = ln(f) / dt, which injects
    2 A E_f.  Returns the rescaled velocity and f."""
    ef = forced_energy(uh, g, kF)
    f = math.sqrt(Ef0 / ef) if ef > 1e-300 else 1.0
    b = band(g, kF)
    return np.array([np.where(b, f * uh[c], uh[c]) for c in range(3)]), f


def forcing_amplitude(uh, g: Grid, p: Params) -> float:
    """A of Eq. 1 for constant-power forcing: A u_hat on the band injects
    2 A E_f = eps_inj per unit time.  A = 0 when the band holds no energy."""
    if p.forcing != FORCE_CONST_POWER:
        return 0.0
    ef = forced_energy(uh, g, p.kF)
    return p.eps_inj / (2.0 * ef) if ef > 1e-300 else 0.0


# --------------------------------------------------------------------------
# Right-hand sides (Eqs. 7-8) and the time integrators (section 2.2)
# --------------------------------------------------------------------------

def rhs_nonlinear(uh, ph, g: Grid, p: Params):
    """N(u, phi): every term of Eqs. 7-8 except -nu|k|^2 u and -D|k|^2 phi.

    du/dt  = P(u x omega)_hat + A u_hat 1[0<|k|^2<=kF^2]
    dphi/dt = -(u.grad phi)_hat - beta u2_hat            (Eq. 8)"""
    A = forcing_amplitude(uh, g, p)
    nl = nonlinear_convective(uh, g) if p.nonlinear_form == NL_CONVECTIVE else nonlinear_rotational(uh, g)
    b = band(g, p.kF)
    ru = [nl[c] + np.where(b, A * uh[c], 0.0) for c in range(3)]
    if p.scalar_on:
        rp = -scalar_advection(uh, ph, g) - p.beta * uh[1]
    else:
        rp = np.zeros_like(ph)
    return ru, rp


def linear_rates(g: Grid, p: Params):
    """Diagonal linear operators: -nu|k|^2 (Eq. 7) and -D|k|^2 (Eq. 8)."""
    k2 = g.k2.astype(np.float64)
    return -p.nu * k2, -p.D * k2


def step_ifrk4(uh, ph, g: Grid, p: Params, dt: float):
    """One Lawson integrating-factor RK4 step.  With E = exp(L dt/2):
      k1 = N(u_n)
      k2 = N(E (u_n + dt/2 k1))
      k3 = N(E u_n + dt/2 k2)
      k4 = N(E^2 u_n + dt E k3)
      u_{n+1} = E^2 u_n + dt/6 (E^2 k1 + 2 E k2 + 2 E k3 + k4)
    applied jointly to (u, phi), each with its own L."""
    Lu, Lp = linear_rates(g, p)
    Eu, Ep = np.exp(0.5 * dt * Lu), np.exp(0.5 * dt * Lp)

    def comb(fu, fp):
        return [fu(c, Eu) for c in range(3)], fp(Ep)

    k1u, k1p = rhs_nonlinear(uh, ph, g, p)
    u2, p2 = comb(lambda c, E: E * (uh[c] + 0.5 * dt * k1u[c]),
                  lambda E: E * (ph + 0.5 * dt * k1p))
    k2u, k2p = rhs_nonlinear(u2, p2, g, p)
    u3, p3 = comb(lambda c, E: E * uh[c] + 0.5 * dt * k2u[c],
                  lambda E: E * ph + 0.5 * dt * k2p)
    k3u, k3p = rhs_nonlinear(u3, p3, g, p)
    u4, p4 = comb(lambda c, E: E * E * uh[c] + dt * E * k3u[c],
                  lambda E: E * E * ph + dt * E * k3p)
    k4u, k4p = rhs_nonlinear(u4, p4, g, p)
    un = [Eu * Eu * uh[c] + dt / 6.0 * (Eu * Eu * k1u[c] + 2 * Eu * k2u[c]
                                        + 2 * Eu * k3u[c] + k4u[c]) for c in range(3)]
    pn = Ep * Ep * ph + dt / 6.0 * (Ep * Ep * k1p + 2 * Ep * k2p + 2 * Ep * k3p + k4p)
    return np.array(un), pn


def step_rk4(uh, ph, g: Grid, p: Params, dt: float):
    """One classical explicit RK4 step with the viscous/diffusive terms inside
    the right-hand side, as the paper integrates Eqs. 7-8 (section 2.2)."""
    Lu, Lp = linear_rates(g, p)

    def full(u, ph_):
        ru, rp = rhs_nonlinear(u, ph_, g, p)
        return [ru[c] + Lu * u[c] for c in range(3)], rp + Lp * ph_

    k1u, k1p = full(uh, ph)
    k2u, k2p = full([uh[c] + 0.5 * dt * k1u[c] for c in range(3)], ph + 0.5 * dt * k1p)
    k3u, k3p = full([uh[c] + 0.5 * dt * k2u[c] for c in range(3)], ph + 0.5 * dt * k2p)
    k4u, k4p = full([uh[c] + dt * k3u[c] for c in range(3)], ph + dt * k3p)
    un = [uh[c] + dt / 6.0 * (k1u[c] + 2 * k2u[c] + 2 * k3u[c] + k4u[c]) for c in range(3)]
    pn = ph + dt / 6.0 * (k1p + 2 * k2p + 2 * k3p + k4p)
    return np.array(un), pn


def step(uh, ph, g: Grid, p: Params, dt: float):
    if p.integrator == INTEG_RK4:
        return step_rk4(uh, ph, g, p, dt)
    return step_ifrk4(uh, ph, g, p, dt)


# --------------------------------------------------------------------------
# CFL (Eq. 10)
# --------------------------------------------------------------------------

def max_abs_sum(uh, g: Grid) -> float:
    """max over the grid of |u1| + |u2| + |u3|."""
    u = velocity(uh, g)
    return float(np.max(np.abs(u[0]) + np.abs(u[1]) + np.abs(u[2])))


def cfl_number(uh, g: Grid, dt: float) -> float:
    """CFL = dt/dx max(|u1|+|u2|+|u3|)  (Eq. 10)."""
    return dt / g.dx * max_abs_sum(uh, g)


def cfl_dt(uh, g: Grid, cfl: float) -> float:
    """The time step that puts Eq. 10 exactly at the target CFL number."""
    m = max_abs_sum(uh, g)
    return cfl * g.dx / m


# --------------------------------------------------------------------------
# Statistics: shell spectra, Table 1, Eqs. 11-13
# --------------------------------------------------------------------------

def shell_index(g: Grid) -> np.ndarray:
    """Shell number n = floor(|k| + 1/2) of every stored mode."""
    return np.floor(np.sqrt(g.k2.astype(np.float64)) + 0.5).astype(np.int64)


def num_shells(N: int, dealias: int = DEALIAS_TWO_THIRDS) -> int:
    """Shells n = 0 .. floor(|k|_max + 1/2) of the retained set."""
    if dealias == DEALIAS_PHASE_SHIFT:
        K = sphere_halfwidth(N)
        return int(math.floor(math.sqrt(float(K * K)) + 0.5)) + 2
    K = (N - 1) // 3
    return int(math.floor(math.sqrt(3.0 * K * K) + 0.5)) + 1


def shell_sum(vals: np.ndarray, g: Grid) -> np.ndarray:
    """Sum a per-mode quantity (already weighted) over each shell n."""
    n = np.broadcast_to(shell_index(g), g.shape_hat)
    v = np.where(g.mask, vals, 0.0)
    return np.bincount(n.ravel(), weights=np.broadcast_to(v, g.shape_hat).ravel(),
                       minlength=num_shells(g.N, g.dealias))[: num_shells(g.N, g.dealias)]


def spectra(uh, ph, g: Grid):
    """Radial energy spectrum E(n) = sum_shell w |u_hat|^2/(2N^6) (Fig. 2b;
    sum_n E(n) = K of Table 1) and the scalar spectrum E_phi(n) with
    sum_n E_phi(n) = <phi^2>/2."""
    n6 = float(g.N) ** 6
    eu = g.w * sum(np.abs(uh[c]) ** 2 for c in range(3)) / (2.0 * n6)
    ep = g.w * np.abs(ph) ** 2 / (2.0 * n6)
    return shell_sum(eu, g), shell_sum(ep, g)


def _moments(a: np.ndarray):
    m2 = float(np.mean(a ** 2))
    m3 = float(np.mean(a ** 3))
    m4 = float(np.mean(a ** 4))
    skew = m3 / m2 ** 1.5 if m2 > 0 else 0.0
    flat = m4 / m2 ** 2 if m2 > 0 else 0.0
    return m2, skew, flat


def stats(uh, ph, g: Grid, p: Params, t: float = 0.0, dt: float | None = None,
          A_hold: float = 0.0) -> dict:
    """One statistics record of the current state (section 2.3).

    Table 1: K = <u.u>/2, eps = 2 nu <S:S>, eta = (nu^3/eps)^(1/4),
    u_rms = sqrt(2K/3), lambda = u_rms sqrt(15 nu/eps), Re_lambda = lambda u_rms/nu,
    l0 = u_rms^3/eps, T_e = l0/u_rms.  Eqs. 11-12: skewness and flatness of
    du_i/dx_i and of dphi/dx_i.  Eq. 13: <phi^2>, production -2 beta <phi u2>
    and chi = 2 D <grad phi . grad phi>.  eps and chi are formed both from the
    spectrum and from grid averages; they agree for dealiased fields.
    With the deterministic forcing, A is the rate of the last step's band
    rescaling (A_hold, 0 before the first step)."""
    if dt is None:
        dt = p.dt
    N = g.N
    n6 = float(N) ** 6
    E, Ephi = spectra(uh, ph, g)
    k2 = g.k2.astype(np.float64)
    msk = g.mask
    eu = g.w * sum(np.abs(uh[c]) ** 2 for c in range(3)) / (2.0 * n6)
    ep = g.w * np.abs(ph) ** 2 / (2.0 * n6)
    Kspec = float(np.sum(E))
    eps = 2.0 * p.nu * float(np.sum(np.where(msk, k2 * eu, 0.0)))
    chi = 2.0 * p.D * 2.0 * float(np.sum(np.where(msk, k2 * ep, 0.0)))
    prod = -2.0 * p.beta * float(np.sum(np.where(msk, g.w * np.real(np.conj(ph) * uh[1]), 0.0))) / n6

    u = velocity(uh, g)
    grads = [[inv(c, N) for c in grad_hat(uh[i], g)] for i in range(3)]  # grads[i][j] = du_i/dx_j
    SS = 0.0
    for i in range(3):
        for j in range(3):
            s = 0.5 * (grads[i][j] + grads[j][i])
            SS += float(np.mean(s * s))
    eps_phys = 2.0 * p.nu * SS
    om = [inv(c, N) for c in curl_hat(uh, g)]
    enst = float(np.mean(om[0] ** 2 + om[1] ** 2 + om[2] ** 2))
    phi = inv(ph, N)
    gp = [inv(c, N) for c in grad_hat(ph, g)]
    chi_phys = 2.0 * p.D * float(np.mean(gp[0] ** 2 + gp[1] ** 2 + gp[2] ** 2))
    skew, flat, skew_phi, flat_phi = [], [], [], []
    for i in range(3):
        _, s_, f_ = _moments(grads[i][i])
        skew.append(s_)
        flat.append(f_)
        _, s_, f_ = _moments(gp[i])
        skew_phi.append(s_)
        flat_phi.append(f_)
    urms = math.sqrt(2.0 * Kspec / 3.0)
    eta = (p.nu ** 3 / eps) ** 0.25 if eps > 0 else float("inf")
    lam = urms * math.sqrt(15.0 * p.nu / eps) if eps > 0 else float("inf")
    l0 = urms ** 3 / eps if eps > 0 else float("inf")
    umax = float(np.max(np.abs(u[0]) + np.abs(u[1]) + np.abs(u[2])))
    A = A_hold if p.forcing == FORCE_HOLD_ENERGY else forcing_amplitude(uh, g, p)
    Ef = forced_energy(uh, g, p.kF)
    return dict(
        t=t, dt=dt, K=Kspec, K_phys=0.5 * float(np.mean(u[0] ** 2 + u[1] ** 2 + u[2] ** 2)),
        eps=eps, eps_phys=eps_phys, enstrophy=enst, eta=eta,
        Re_lambda=lam * urms / p.nu if eps > 0 else float("inf"),
        Te=l0 / urms if urms > 0 else float("inf"), urms=urms, lam=lam, l0=l0,
        cfl=dt / g.dx * umax, umax=umax,
        kmax_eta=(N / 3.0) * eta, kmax_eta_sqrt2=(math.sqrt(2.0) * N / 3.0) * eta,
        skew=skew, flat=flat,
        phi_var=float(np.mean(phi ** 2)), phi_prod=prod,
        phi_prod_phys=-2.0 * p.beta * float(np.mean(phi * u[1])),
        chi=chi, chi_phys=chi_phys, skew_phi=skew_phi, flat_phi=flat_phi,
        A=A, E_forced=Ef, P_inj=2.0 * A * Ef, E=E, Ephi=Ephi)


# --------------------------------------------------------------------------
# Initial condition (section 2.3: Rogallo-type isotropic solenoidal field)
# --------------------------------------------------------------------------

_GAMMA = 0x9E3779B97F4A7C15
_M64 = (1 << 64) - 1


def splitmix64(seed: int, i):
    """Element i (0-based) of the SplitMix64 stream seeded with ``seed``
    (Steele, Lea and Flood, OOPSLA 2014): mix(seed + (i+1) * gamma mod 2^64).
    Works on Python ints or uint64 NumPy arrays."""
    if isinstance(i, np.ndarray):
        with np.errstate(over="ignore"):
            z = np.uint64(seed & _M64) + (i.astype(np.uint64) + np.uint64(1)) * np.uint64(_GAMMA)
            z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
            z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
            return z ^ (z >> np.uint64(31))
    z = (seed + (i + 1) * _GAMMA) & _M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
    return z ^ (z >> 31)


def uniform01(seed: int, i):
    """(0, 1] uniform from the top 53 bits of a SplitMix64 draw."""
    x = splitmix64(seed, i)
    if isinstance(x, np.ndarray):
        return ((x >> np.uint64(11)).astype(np.float64) + 1.0) * 2.0 ** -53
    return ((x >> 11) + 1) * 2.0 ** -53


def mode_key(kx, ky, kz):
    """Grid-independent 36-bit key of a wavevector (|k_i| < 2048)."""
    return ((kx + 2048) << 24) | ((ky + 2048) << 12) | (kz + 2048)


def target_shell_energy(nmax: int, shape: int, K0: float, kF: float) -> np.ndarray:
    """Target E(n), n = 0..nmax-1, normalised so that sum_n E(n) = K0.
    shape IC_SPECTRUM_K4: n^4 exp(-2 (n/4)^2); IC_PAPER_EQ9: Eq. 9's
    (n/kF)^2 for n <= kF and (n/kF)^(-5/3) above.  E(0) = 0."""
    n = np.arange(nmax, dtype=np.float64)
    if shape == IC_PAPER_EQ9:
        safe = np.maximum(n, 1.0)
        e = np.where(n <= kF, (n / kF) ** 2, (safe / kF) ** (-5.0 / 3.0))
    else:
        e = n ** 4 * np.exp(-2.0 * (n / 4.0) ** 2)
    e[0] = 0.0
    return K0 * e / np.sum(e)


def ic_random(g: Grid, seed: int, K0: float, shape: int = IC_SPECTRUM_K4,
              kF: float = 2.0) -> np.ndarray:
    """Random-phase isotropic solenoidal velocity with a prescribed shell spectrum.

    For every stored mode k != 0 with kx > 0, or kx = 0 and (ky, kz) > (0, 0)
    lexicographically, each component draws one complex Gaussian
    sqrt(-2 ln u1) exp(2 pi i u2) (Box-Muller) from SplitMix64 elements
    8*key + 2c and 8*key + 2c + 1.  The vector is projected onto the plane
    normal to k, the remaining kx = 0 modes take the conjugate of their partner
    (real field), and every shell is rescaled so that E(n) equals the target."""
    N, K = g.N, g.K
    kx, ky, kz = np.broadcast_arrays(g.kx, g.ky, g.kz)
    canon = (kx > 0) | ((kx == 0) & ((ky > 0) | ((ky == 0) & (kz > 0))))
    # Draw for the canonical wavevector of each stored mode (the partner for
    # non-canonical kx = 0 modes), then conjugate there.
    cx = np.where(canon, kx, -kx)
    cy = np.where(canon, ky, -ky)
    cz = np.where(canon, kz, -kz)
    key = mode_key(cx.astype(np.int64), cy.astype(np.int64), cz.astype(np.int64)).astype(np.uint64)
    z = []
    for c in range(3):
        u1 = uniform01(seed, key * np.uint64(8) + np.uint64(2 * c))
        u2 = uniform01(seed, key * np.uint64(8) + np.uint64(2 * c + 1))
        r = np.sqrt(-2.0 * np.log(u1))
        z.append(r * np.cos(2.0 * np.pi * u2) + 1j * r * np.sin(2.0 * np.pi * u2))
    # Project with the canonical wavevector, then conjugate the partners.
    kc = (cx, cy, cz)
    k2c = (cx ** 2 + cy ** 2 + cz ** 2).astype(np.float64)
    k2s = np.where(k2c == 0, 1.0, k2c)
    kdz = sum(kc[i] * z[i] for i in range(3))
    z = [z[i] - kc[i] * kdz / k2s for i in range(3)]
    z = [np.where(canon, zc, np.conj(zc)) for zc in z]
    keep = g.mask & (g.k2 > 0)
    z = np.array([np.where(keep, zc, 0.0) for zc in z])
    # Per-shell rescale to the target spectrum.
    n6 = float(N) ** 6
    raw = shell_sum(g.w * np.sum(np.abs(z) ** 2, axis=0) / (2.0 * n6), g)
    tgt = target_shell_energy(len(raw), shape, K0, kF)
    # only shells that hold modes take part in the normalisation
    tgt = np.where(raw > 0, tgt, 0.0)
    tgt = K0 * tgt / np.sum(tgt)
    fac = np.where(raw > 0, np.sqrt(tgt / np.where(raw > 0, raw, 1.0)), 0.0)
    # modes outside the retained set are already zero; clamp their shell index
    n = np.minimum(np.broadcast_to(shell_index(g), g.shape_hat), len(fac) - 1)
    return z * fac[n][None]


def ic_taylor_green(g: Grid, amp: float = 1.0) -> np.ndarray:
    """Taylor-Green vortex u = A (sin x cos y cos z, -cos x sin y cos z, 0),
    sampled on the grid and transformed (K = A^2/8)."""
    ux = amp * np.sin(g.x) * np.cos(g.y) * np.cos(g.z)
    uy = -amp * np.cos(g.x) * np.sin(g.y) * np.cos(g.z)
    uz = np.zeros((g.N, g.N, g.N))
    shape = (g.N, g.N, g.N)
    return np.array([truncate(fwd(np.broadcast_to(a, shape)), g) for a in (ux, uy, uz)])


def init_field(g: Grid, p: Params):
    """Initial (u_hat, phi_hat).  phi_0 = 0 (section 2.3)."""
    if p.ic == IC_TAYLOR_GREEN_NOISE:
        uh = ic_taylor_green(g, 1.0)
        if p.ic_noise_frac > 0:
            uh = uh + ic_random(g, p.seed, p.ic_noise_frac * 0.125, IC_SPECTRUM_K4, p.kF)
    else:
        uh = ic_random(g, p.seed, p.ic_energy, p.ic, p.kF)
    ph = np.zeros(g.shape_hat, dtype=np.complex128)
    return uh, ph


# --------------------------------------------------------------------------
# Driver: records every record_every steps (section 2.3)
# --------------------------------------------------------------------------

def run(p: Params, nsteps: int, uh=None, ph=None, with_records: bool = True):
    """Advance ``nsteps`` steps from the IC (or from the given state).

    With ``cfl > 0`` the step is reset to put Eq. 10 at ``cfl`` at step 0 and
    at every record step, and held in between.  Records are taken of the state
    at every step n with n % record_every == 0 and of the final state.  With
    the deterministic forcing the band energy of the starting state is held
    after every step."""
    g = Grid(p.N, p.dealias)
    if uh is None:
        uh, ph = init_field(g, p)
    dt = p.dt
    t = 0.0
    recs = []
    hold = p.forcing == FORCE_HOLD_ENERGY
    Ef0 = forced_energy(uh, g, p.kF) if hold else 0.0  # the band energy to hold
    A_hold = 0.0
    for n in range(nsteps):
        if n % p.record_every == 0:
            if p.cfl > 0:
                dt = cfl_dt(uh, g, p.cfl)
            if with_records:
                recs.append(dict(step=n, **stats(uh, ph, g, p, t, dt, A_hold)))
        uh, ph = step(uh, ph, g, p, dt)
        if hold:
            uh, f = hold_band_energy(uh, g, p.kF, Ef0)
            A_hold = math.log(f) / dt
        t += dt
    if with_records:
        recs.append(dict(step=nsteps, **stats(uh, ph, g, p, t, dt, A_hold)))
    return uh, ph, recs, t, dt


# --------------------------------------------------------------------------
# Direct triad sums for sparse states (any N)
# --------------------------------------------------------------------------

def rhs_sparse_triads(modes, N: int, p: Params):
    """N(u, phi) of a state with few non-zero modes, by direct summation.

    ``modes`` maps retained (kx, ky, kz), kx >= 0, to (u1, u2, u3, phi)
    unnormalised coefficients; kx = 0 entries must come in conjugate pairs.
    The retained set is the 2/3 cube |k_i| <= (N-1)//3, or with
    ``p.dealias`` = DEALIAS_PHASE_SHIFT the sphere 9|k|^2 < 2 N^2 (section
    2.3).  With u(x) = N^-3 sum_p u_p exp(i p.x) (Eq. 5), the dealiased
    products of retained modes are alias-free on the retained set (2/3 rule:
    every alias lands outside the cube; phase shifts: aliases wrapped in one
    direction cancel between the two grids and the rest land outside the
    sphere), so

        (u x omega)_k   = N^-3 sum_{p+q=k} u_p x (i q x u_q)
        (u.grad phi)_k  = N^-3 sum_{p+q=k} (u_p . i q) phi_q

    over the full (conjugate-completed) mode set.  Returns a dict over the
    output modes k (kx >= 0, |k_i| <= K) that receive a contribution or carry
    forcing/source terms: k -> (r1, r2, r3, r_phi) as in rhs_nonlinear."""
    sphere = p.dealias == DEALIAS_PHASE_SHIFT
    K = sphere_halfwidth(N) if sphere else (N - 1) // 3
    full = {}
    for (kx, ky, kz), v in modes.items():
        v = np.asarray(v, dtype=np.complex128)
        full[(kx, ky, kz)] = v
        if kx > 0:
            full[(-kx, -ky, -kz)] = np.conj(v)
    keys = list(full)
    kv = np.array(keys, dtype=np.int64)
    vals = np.array([full[k] for k in keys])
    # forcing amplitude from the band energy of the stored half
    A = 0.0
    if p.forcing == FORCE_CONST_POWER:
        s = 0.0
        for (kx, ky, kz), v in modes.items():
            k2 = kx * kx + ky * ky + kz * kz
            if 0 < k2 <= p.kF * p.kF:
                s += (1.0 if kx == 0 else 2.0) * float(np.sum(np.abs(v[:3]) ** 2))
        ef = s / (2.0 * float(N) ** 6)
        A = p.eps_inj / (2.0 * ef) if ef > 1e-300 else 0.0
    acc_u, acc_s = {}, {}
    for a in range(len(keys)):
        pvec = kv[a]
        up = vals[a][:3]
        for b in range(len(keys)):
            q = kv[b]
            k = pvec + q
            if k[0] < 0 or np.any(np.abs(k) > K) or (sphere and 9 * int(k @ k) >= 2 * N * N):
                continue
            uq, phq = vals[b][:3], vals[b][3]
            om = 1j * np.cross(q.astype(np.float64), uq)
            kk = tuple(int(c) for c in k)
            acc_u[kk] = acc_u.get(kk, 0) + np.cross(up, om)
            acc_s[kk] = acc_s.get(kk, 0) + np.dot(up, 1j * q.astype(np.float64)) * phq
    out = {}
    n3 = float(N) ** 3
    for kk in set(acc_u) | set(modes):
        k = np.array(kk, dtype=np.float64)
        k2 = float(k @ k)
        nl = np.asarray(acc_u.get(kk, np.zeros(3, dtype=complex)), dtype=np.complex128) / n3
        if k2 > 0:
            nl = nl - k * (k @ nl) / k2
        else:
            nl = np.zeros(3, dtype=np.complex128)
        v = np.asarray(modes.get(kk, np.zeros(4, dtype=complex)), dtype=np.complex128)
        if 0 < k2 <= p.kF * p.kF:
            nl = nl + A * v[:3]
        sh = complex(acc_s.get(kk, 0.0)) / n3
        rp = (-sh - p.beta * v[1]) if p.scalar_on else 0.0
        out[kk] = np.array([nl[0], nl[1], nl[2], rp], dtype=np.complex128)
    return out


# --------------------------------------------------------------------------
# Direct sums for separable states (any N): fields that are sums of products
# of one-dimensional factors
# --------------------------------------------------------------------------

class SeparableRHS:
    """N(u, phi) of Eqs. 7-8 (2/3 rule, rotational form, no linear terms) for a
    state whose fields are sums of products of 1D factors, at grids too large
    for the FFT oracle.

    A field f(x) = N^-3 sum_k f_k exp(i k.x) with f_k = sum_t X_t(kx) Y_t(ky)
    Z_t(kz) is a sum of products a(x1) b(x2) c(x3).  The dealiased product of
    two such fields keeps, by the definition of the 2/3 rule's alias-free
    products, (fg)_k = N^-3 sum_{p+q=k} f_p g_q for |k_i| <= K, and for one term
    of each that sum factorises into three 1D convolutions:
        (fg)_k = [N^-1 (X * X')(kx)] [N^-1 (Y * Y')(ky)] [N^-1 (Z * Z')(kz)],
    each restricted to |k| <= K (the cube truncation acts per axis).  Spectral
    derivatives multiply one factor by i k.  So u x omega and u.grad phi are
    sums of products of 1D factors, and any plane kz of the output is a small
    matrix product; projection, forcing and the scalar source are applied on
    the plane as in ``rhs_nonlinear``.

    ``u_factors`` (3 fields) and ``phi_factors`` are lists of (X, Y, Z) arrays
    over k = -K..K (index k + K), conjugate-symmetric (real fields)."""

    def __init__(self, u_factors, phi_factors, N: int, p: Params):
        self.N, self.p = N, p
        self.K = K = (N - 1) // 3
        self.k = np.arange(-K, K + 1)
        u = [[tuple(np.asarray(a, dtype=np.complex128) for a in t) for t in f] for f in u_factors]
        ph = [tuple(np.asarray(a, dtype=np.complex128) for a in t) for t in phi_factors]
        self.u = u

        def d(terms, axis):  # derivative along x_{axis+1}: i k on that factor
            return [tuple(1j * self.k * a if i == axis else a for i, a in enumerate(t)) for t in terms]

        def neg(terms):
            return [(-t[0], t[1], t[2]) for t in terms]

        # omega = curl u: (d2 u3 - d3 u2, d3 u1 - d1 u3, d1 u2 - d2 u1)
        w = [d(u[2], 1) + neg(d(u[1], 2)), d(u[0], 2) + neg(d(u[2], 0)), d(u[1], 0) + neg(d(u[0], 1))]
        self.nl = [self._mul(u[1], w[2]) + neg(self._mul(u[2], w[1])),
                   self._mul(u[2], w[0]) + neg(self._mul(u[0], w[2])),
                   self._mul(u[0], w[1]) + neg(self._mul(u[1], w[0]))]
        self.s = sum((self._mul(u[i], d(ph, i)) for i in range(3)), [])
        # constant-power forcing amplitude from the band energy (section 2.3)
        self.A = 0.0
        if p.forcing == FORCE_CONST_POWER:
            kb = int(math.floor(p.kF))
            s_ = 0.0
            for kz in range(-kb, kb + 1):
                for ky in range(-kb, kb + 1):
                    for kx in range(0, kb + 1):
                        k2 = kx * kx + ky * ky + kz * kz
                        if 0 < k2 <= p.kF * p.kF and max(kx, abs(ky), abs(kz)) <= K:
                            w_ = 1.0 if kx == 0 else 2.0
                            s_ += w_ * sum(abs(self._at(u[c], kx, ky, kz)) ** 2 for c in range(3))
            ef = s_ / (2.0 * float(N) ** 6)
            self.A = p.eps_inj / (2.0 * ef) if ef > 1e-300 else 0.0

    def _mul(self, fa, fb):
        """Terms of the dealiased product of two separable fields."""
        K, N = self.K, self.N
        out = []
        for ta in fa:
            for tb in fb:
                out.append(tuple(np.convolve(a, b)[K:3 * K + 1] / N for a, b in zip(ta, tb)))
        return out

    def _at(self, terms, kx, ky, kz):
        K = self.K
        return sum(t[0][kx + K] * t[1][ky + K] * t[2][kz + K] for t in terms)

    def _plane(self, terms, kz):
        """Dense [ky+K][kx] values (kx >= 0) of a separable field at one kz."""
        K = self.K
        X = np.array([t[0][K:] for t in terms])          # (T, K+1)
        Y = np.array([t[1] for t in terms])              # (T, 2K+1)
        Z = np.array([t[2][kz + K] for t in terms])      # (T,)
        return (Y.T * Z) @ X

    def plane(self, kz: int) -> np.ndarray:
        """The right-hand side (r1, r2, r3, r_phi) at one kz, compact layout
        [f][ky+K][kx]."""
        K, p = self.K, self.p
        kx = np.arange(0, K + 1)[None, :]
        ky = np.arange(-K, K + 1)[:, None]
        kzv = float(kz)
        nl = [self._plane(t, kz) for t in self.nl]
        k2 = (kx * kx + ky * ky + kz * kz).astype(np.float64)
        # Leray projection (Eq. 7); k = 0 carries no velocity
        kd = (kx * nl[0] + ky * nl[1] + kzv * nl[2]) / np.where(k2 == 0, 1.0, k2)
        nl = [nl[0] - kx * kd, nl[1] - ky * kd, nl[2] - kzv * kd]
        nl = [np.where(k2 == 0, 0.0, c) for c in nl]
        u2 = self._plane(self.u[1], kz)
        bandm = (k2 > 0) & (k2 <= p.kF * p.kF)
        if p.forcing == FORCE_CONST_POWER:
            for c in range(3):
                nl[c] = nl[c] + np.where(bandm, self.A * self._plane(self.u[c], kz), 0.0)
        if p.scalar_on:
            rp = -self._plane(self.s, kz) - p.beta * u2
        else:
            rp = np.zeros_like(u2)
        return np.array(nl + [rp])
