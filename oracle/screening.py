"""FP64 oracle: model dielectric functions and the screened loss function.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper compares the loss function built from the RPA dielectric function
with screened forms that keep Im eps from the calculation and take |eps| from
a model (Section IV.C):

  screened loss      Im(-1/eps)_scr = Im eps(w, q) / |eps_scr(w, q)|^2        (Eq. (ELF_screening))
  modified Thomas-Fermi model (Eq. (MTF)):
      eps_MTF = 1 + [1/(eps0 - 1) + tau (q/q_TF)^2 + q^4/(4 m_e^2 w_p^2) - (w/w_p)^2]^-1
  Lindhard model of a homogeneous electron gas (Eq. (Lindhard)):
      eps_L = 1 + 3 w_p^2/(q^2 v_F^2) (1/2 + F_+ + F_-),
      F_pm = q_F/(4 q) (1 - Q_pm^2) Log[(Q_pm + 1)/(Q_pm - 1)],
      Q_pm = q/(2 q_F) pm w/(q v_F) pm i f_p w_p/(q v_F),
  with q_F = (3 pi^2 n_e)^(1/3), v_F = q_F/m_e, w_p = sqrt(4 pi alpha n_e/m_e)
  (Log is the principal branch of the complex logarithm).

Everything here is in natural units: energies and momenta in eV (hbar = c = 1),
the electron density n_e in eV^3.
"""
from __future__ import annotations

import cmath
from math import pi, sqrt

ALPHA = 1.0 / 137.035999084
ME_EV = 510998.95000


def eps_mtf(w, q, eps0, tau, wp, qtf, me=ME_EV):
    """Modified Thomas-Fermi dielectric function (real) at energy w and momentum q (eV)."""
    d = 1.0 / (eps0 - 1.0) + tau * (q / qtf) ** 2 + q ** 4 / (4.0 * me * me * wp * wp) - (w / wp) ** 2
    return 1.0 + 1.0 / d


def electron_gas(ne, me=ME_EV):
    """(q_F, v_F, w_p) of a homogeneous electron gas of density ne (eV^3)."""
    qf = (3.0 * pi * pi * ne) ** (1.0 / 3.0)
    return qf, qf / me, sqrt(4.0 * pi * ALPHA * ne / me)


def eps_lindhard(w, q, ne, fp, me=ME_EV):
    """Lindhard dielectric function (complex) with the damping f_p w_p of the paper."""
    qf, vf, wp = electron_gas(ne, me)
    a = q / (2.0 * qf)
    b = (w + 1j * fp * wp) / (q * vf)
    total = 0.5
    for Q in (a + b, a - b):
        total += qf / (4.0 * q) * (1.0 - Q * Q) * cmath.log((Q + 1.0) / (Q - 1.0))
    return 1.0 + 3.0 * wp * wp / (q * q * vf * vf) * total


def screened_loss(eps, eps_scr):
    """Im eps / |eps_scr|^2."""
    return eps.imag / abs(eps_scr) ** 2
