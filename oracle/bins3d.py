"""FP64 oracle: the composite dielectric function binned in three-dimensional
momentum space, the filling of empty bins, and the isotropic loss function.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Section III (the paragraphs around Eq. (e_comp)) describes the step that turns
the per-q results into the tables the rate uses:

* the composite function takes eps^LFE(w, q+G) = 1/[eps^-1]_GG (Eq. (eps_LFE))
  for |q+G| <= q_LFE and eps^noLFE(w, q+G) = eps_GG (Eq. (eps_noLFE)) above it
  (Eq. (e_comp));
* its values are binned in spherical shells of width dq, each split into
  N_theta polar and N_phi azimuthal cells (the paper: 9, 16 and 0.02 alpha m_e);
* bins left empty are filled by interpolation of the surrounding bins;
* in the isotropic approximation the loss function is averaged over the
  directions of each shell.

Readings (the paper gives no formula for them): a value falls in shell
floor(|k|/dq), polar cell floor(theta N_theta/pi) and azimuthal cell
floor(phi' N_phi/(2 pi)) with phi' = atan2(k_y, k_x) taken in [0, 2 pi) (the
edge values pi and 2 pi go to the last cell); a bin holds the mean of the
complex eps values that fall in it; an empty bin takes the linear interpolation
in |k| (shell centres) between the nearest filled shells of the same angular
cell, and stays empty when no filled shell lies on one side; the isotropic loss
of a shell is the mean over its non-empty angular cells of the loss of each
cell, Im eps_cell / |eps_scr|^2 (Eq. (ELF_screening); eps_scr = eps_cell gives
Im(-1/eps_cell)).
"""
from __future__ import annotations

import numpy as np
from math import atan2, acos, floor, pi, sqrt


def bin_index(k, dq, nshell, nth, nph):
    """(shell, theta cell, phi cell) of a momentum vector k (bohr^-1), or None
    when |k| is zero or past the last shell."""
    kk = sqrt(k[0] * k[0] + k[1] * k[1] + k[2] * k[2])
    if kk <= 0.0:
        return None
    s = int(floor(kk / dq))
    if s >= nshell:
        return None
    th = acos(max(-1.0, min(1.0, k[2] / kk)))
    it = min(nth - 1, int(floor(th * nth / pi)))
    ph = atan2(k[1], k[0])
    if ph < 0.0:
        ph += 2.0 * pi
    ip = min(nph - 1, int(floor(ph * nph / (2.0 * pi))))
    return s, it, ip


def composite_eps(kvec, eps_inv_diag, eps_diag, q_lfe):
    """eps^comp[w][G] of Eq. (e_comp): 1/[eps^-1]_GG where |q+G| <= q_lfe, else eps_GG."""
    kmag = np.linalg.norm(kvec, axis=1)
    return np.where(kmag[None, :] <= q_lfe, 1.0 / eps_inv_diag, eps_diag)


def bin_eps(kvecs, eps_list, dq, nshell, nth, nph):
    """Mean complex eps per (shell, theta, phi, w) over every (q, G) value;
    kvecs: list of [ng][3], eps_list: list of [nw][ng].  Returns (eps, count)."""
    nw = eps_list[0].shape[0]
    tot = np.zeros((nshell, nth, nph, nw), complex)
    cnt = np.zeros((nshell, nth, nph))
    for kv, ev in zip(kvecs, eps_list):
        for g in range(kv.shape[0]):
            b = bin_index(kv[g], dq, nshell, nth, nph)
            if b is None:
                continue
            tot[b] += ev[:, g]
            cnt[b] += 1
    out = np.zeros_like(tot)
    nz = cnt > 0
    out[nz] = tot[nz] / cnt[nz][:, None]
    return out, cnt


def fill_empty(eps, cnt, dq):
    """Empty bins between filled shells of the same angular cell get the linear
    interpolation in |k| of the nearest filled shells on either side (filled
    count set to -1 to mark them); the others stay empty."""
    eps = eps.copy()
    cnt = cnt.copy()
    nshell, nth, nph, _ = eps.shape
    for it in range(nth):
        for ip in range(nph):
            filled = [s for s in range(nshell) if cnt[s, it, ip] > 0]
            for a, b in zip(filled[:-1], filled[1:]):
                for s in range(a + 1, b):
                    x = (s - a) / (b - a)          # shell centres are equally spaced
                    eps[s, it, ip] = (1.0 - x) * eps[a, it, ip] + x * eps[b, it, ip]
                    cnt[s, it, ip] = -1
    return eps, cnt


def isotropic_loss(eps, cnt, eps_scr=None):
    """L[shell][w] = mean over the non-empty angular cells (count != 0) of
    Im eps_cell / |eps_scr|^2, with eps_scr = eps_cell when eps_scr is None, else
    eps_scr[shell][w] (a model evaluated at the shell centre).  Shells without a
    non-empty cell give 0.  Returns (L, number of cells used per shell)."""
    nshell, nth, nph, nw = eps.shape
    L = np.zeros((nshell, nw))
    ncell = np.zeros(nshell)
    for s in range(nshell):
        for it in range(nth):
            for ip in range(nph):
                if cnt[s, it, ip] == 0:
                    continue
                e = eps[s, it, ip]
                den = np.abs(e) ** 2 if eps_scr is None else np.abs(eps_scr[s]) ** 2
                L[s] += e.imag / den
                ncell[s] += 1
        if ncell[s] > 0:
            L[s] /= ncell[s]
    return L, ncell
