"""Kinetic equations of the photon/pair cascade (Eq. 9-10): a CPU solver used
as a statistical oracle for the Monte-Carlo step.

TEST INFRASTRUCTURE: only tests/ (and nothing on the product path) use this.

Setting of the paper's validation test (section 4): electrons, positrons
and photons moving in the plane perpendicular to a constant magnetic field
b0 (normalised units).  Every particle then has chi proportional to its
momentum: chi = |p| b0 / a_S for a lepton, chi_gamma = gamma_gamma b0 / a_S
for a photon (Eq. 1 with E = 0 and k perpendicular to B), so Eq. 9-10 close
on the energy distributions f_-, f_+, f_gamma alone:

  d f_gamma / dt = [photons emitted by e- and e+ at gamma_gamma]
                   - W_pm(gamma_gamma) f_gamma                               (Eq. 9)
  d f_pm / dt    = - W_gamma(gamma) f_pm + [leptons recoiling into gamma]
                   + [leptons created at gamma by photon decay]             (Eq. 10)

with the emission spectrum d2N/dt du = C F_gamma(u; chi)/gamma (Eq. 2, u =
gamma_gamma/gamma) and the pair spectrum d2N/dt dv = C F_pm(v; chi_gamma)/
gamma_gamma (Eq. 3, v = gamma_-/gamma_gamma), C = alpha/(sqrt(3) pi tau_c w).
Readings (listed with the others of the method): the photon loss term of
Eq. 9 removes each decaying photon once (its printed factor 2 counts the two
leptons created); the recoiling lepton keeps |p| - u gamma (collinear,
momentum conserving, as in Eq. 8), and the pair leptons get v gamma_gamma and
(1 - v) gamma_gamma of momentum along k (the Monte-Carlo step's choices);
photons of every energy radiate into f_gamma (the Monte-Carlo step stores only
those above photon_min_gamma and counts the energy of the others), and only
photons above 2 m c^2 decay (section 2).

Discretisation: log grids of lepton momentum and photon energy; particles
are numbers per bin at the bin's centre; a transition to a value between two
centres is shared between them so that both the number and the value
(momentum, photon energy) are conserved; the rates come from a quadrature of
the spectra over the logit of u (or v) with the oracle's own Bessel functions
(or_F_gamma, or_F_pair).  dN/dt = A N is linear with constant coefficients
(chi depends only on the bin), so N(t) = expm(A t) N(0).
"""
from __future__ import annotations

import math

import numpy as np

from . import F_gamma, F_pair, units


def _log_grid(lo, hi, n):
    edges = np.exp(np.linspace(math.log(lo), math.log(hi), n + 1))
    return np.sqrt(edges[:-1] * edges[1:])


def _deposit(centres, x):
    """Indices and weights sharing the values x between neighbouring centres
    (number and value conserved; clamped at the ends)."""
    x = np.asarray(x, dtype=float)
    i = np.searchsorted(centres, x) - 1
    i = np.clip(i, 0, len(centres) - 2)
    c0, c1 = centres[i], centres[i + 1]
    w1 = np.clip((x - c0) / (c1 - c0), 0.0, 1.0)
    below = x <= centres[0]
    w1 = np.where(below, 0.0, w1)
    above = x >= centres[-1]
    i = np.where(above, len(centres) - 2, i)
    w1 = np.where(above, 1.0, w1)
    return i, 1.0 - w1, w1


class Cascade:
    """Kinetic model of e-, e+ and photons in a constant field b0."""

    def __init__(self, b0: float, p_max: float = 4400.0, n_lep: int = 260, n_pho: int = 320,
                 pho_min: float = 1e-4, n_quad: int = 480, lambda_m: float = 0.8e-6,
                 pairs: bool = True):
        self.U = units(lambda_m)
        self.b0 = b0
        self.p = _log_grid(0.05, p_max, n_lep)          # lepton momentum centres
        self.g = np.sqrt(1.0 + self.p ** 2)             # lepton gamma
        self.k = _log_grid(pho_min, p_max, n_pho)       # photon energy centres
        self.chi_l = self.p * b0 / self.U.a_S
        self.chi_k = self.k * b0 / self.U.a_S
        L, G = n_lep, n_pho
        self.L, self.G = L, G
        n = 2 * L + G
        A = np.zeros((n, n))
        s = np.linspace(-26.0, 14.0, n_quad)            # logit nodes of u (and v)
        ds = s[1] - s[0]
        u = 1.0 / (1.0 + np.exp(-s))
        omu = 1.0 / (1.0 + np.exp(s))
        wq = u * omu * ds                               # du = u (1 - u) ds
        wq[0] *= 0.5
        wq[-1] *= 0.5
        C = self.U.C_rate
        self.W_emit = np.zeros(L)
        for j in range(L):
            rate = C * F_gamma(u, self.chi_l[j], omu) * wq / self.g[j]   # per unit u-mass
            rate = np.maximum(rate, 0.0)
            self.W_emit[j] = rate.sum()
            gg = u * self.g[j]
            prec = np.maximum(self.p[j] - gg, 0.0)       # recoil: |p| - u gamma
            ki, kw0, kw1 = _deposit(self.k, gg)
            li, lw0, lw1 = _deposit(self.p, prec)
            for sp in (0, 1):                           # e- block, e+ block
                col = sp * L + j
                A[col, col] -= self.W_emit[j]
                np.add.at(A[:, col], 2 * L + ki, rate * kw0)
                np.add.at(A[:, col], 2 * L + ki + 1, rate * kw1)
                np.add.at(A[:, col], sp * L + li, rate * lw0)
                np.add.at(A[:, col], sp * L + li + 1, rate * lw1)
        self.W_pair = np.zeros(G)
        if pairs:
            for k in range(G):
                if self.k[k] <= 2.0:
                    continue
                rate = C * F_pair(u, self.chi_k[k], omu) * wq / self.k[k]
                rate = np.maximum(rate, 0.0)
                self.W_pair[k] = rate.sum()
                col = 2 * L + k
                A[col, col] -= self.W_pair[k]
                ei, ew0, ew1 = _deposit(self.p, u * self.k[k])
                pi_, pw0, pw1 = _deposit(self.p, omu * self.k[k])
                np.add.at(A[:, col], ei, rate * ew0)
                np.add.at(A[:, col], ei + 1, rate * ew1)
                np.add.at(A[:, col], L + pi_, rate * pw0)
                np.add.at(A[:, col], L + pi_ + 1, rate * pw1)
        self.A = A

    def initial_electrons(self, p0: float, n: float) -> np.ndarray:
        N = np.zeros(2 * self.L + self.G)
        i, w0, w1 = _deposit(self.p, np.array([p0]))
        N[i[0]] += n * w0[0]
        N[i[0] + 1] += n * w1[0]
        return N

    def evolve(self, N0: np.ndarray, times) -> list:
        from scipy.linalg import expm
        out, t_prev, N = [], 0.0, N0.copy()
        for t in times:
            if t > t_prev:
                N = expm(self.A * (t - t_prev)) @ N
            out.append(N.copy())
            t_prev = t
        return out

    def moments(self, N: np.ndarray, photon_min: float = 2.0) -> dict:
        L = self.L
        ne, npos, ng = N[:L], N[L:2 * L], N[2 * L:]
        hi = self.k > photon_min
        return {
            "n_electron": ne.sum(), "n_positron": npos.sum(), "n_photon": ng[hi].sum(),
            "e_electron": (ne * self.g).sum(), "e_positron": (npos * self.g).sum(),
            "e_photon": (ng * self.k).sum(),
            "chi_electron": (ne * self.chi_l).sum() / max(ne.sum(), 1e-300),
        }
