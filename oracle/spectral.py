"""FP64 oracle of the spectral route to chi0 (the paper's Eq. (eRPA_spectral)
with the principal part from the Kramers-Kronig relations).

TEST INFRASTRUCTURE ONLY (see the package docstring): imported by tests/.

Reading.  The spectral part keeps a delta(w - dE_t) per transition.  On a
uniform energy grid E_b = E_0 + b dE the delta is shared between the two grid
points around dE_t with linear (hat) weights, which keeps its zeroth and first
moments exactly.  The spectral weights

    S_b[G][G'] = 2/(N_k V) sum_t phi_b(dE_t) conj(rho_t(G)) rho_t(G')

are formed once per q, not per frequency.  The Kramers-Kronig step, which
gives the principal part from the spectral one, is done with the same retarded
broadening as the direct sum (Eq. (RPA) with W_t(w)),

    chi0(w) = sum_b S_b [1/(w - E_b + i eta) - 1/(w + E_b + i eta)],

so that the route equals the direct sum exactly when every dE_t lies on the
grid, and otherwise differs by the interpolation of W in energy (second order
in dE).
"""
from __future__ import annotations

import numpy as np


def hat_weights(dE, E0, step, nbin):
    """Grid index b and weights (1 - x, x) of every transition on the grid
    E_b = E0 + b step, b = 0..nbin-1: dE = E_b + x step with 0 <= x < 1."""
    u = (np.asarray(dE, float) - E0) / step
    b = np.floor(u).astype(np.int64)
    if np.any(b < 0) or np.any(b > nbin - 2):
        raise ValueError("transition energies outside the grid")
    x = u - b
    return b, 1.0 - x, x


def spectral_weights(rho, dE, E0, step, nbin, nk, vcell):
    """S[b][G][G'] = 2/(nk V) sum_t phi_b(dE_t) conj(rho[t,G]) rho[t,G'] on the grid."""
    pref = 2.0 / (nk * vcell)
    b, w0, w1 = hat_weights(dE, E0, step, nbin)
    ng = rho.shape[1]
    S = np.zeros((nbin, ng, ng), complex)
    for t in range(rho.shape[0]):
        outer = np.outer(rho[t].conj(), rho[t])
        S[b[t]] += w0[t] * outer
        S[b[t] + 1] += w1[t] * outer
    return pref * S


def chi0_from_spectral(S, E0, step, w, eta):
    """chi0[w][G][G'] = sum_b S_b (1/(w - E_b + i eta) - 1/(w + E_b + i eta))."""
    E = E0 + step * np.arange(S.shape[0])
    w = np.asarray(w, float)[:, None]
    K = 1.0 / (w - E[None, :] + 1j * eta) - 1.0 / (w + E[None, :] + 1j * eta)     # [nw][nbin]
    return np.einsum("wb,bgh->wgh", K, S)
