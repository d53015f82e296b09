"""Synthetic-input preparation on the product side.

The path starts from Bloch coefficients (Eq. (RPA) states).  For the seeded
synthetic workloads the raw complex draws Z are turned into S(k)-orthonormal
coefficients C = L^{-H} Q, with S(k) = L L^H from the library's overlap
kernel (qcx_overlap) and Q the orthonormal factor of L^H Z (LAPACK via
numpy).  This is input preparation, outside any timed region.
"""
from __future__ import annotations

import numpy as np


def orthonormalise(S: np.ndarray, Z: np.ndarray) -> np.ndarray:
    """S: [nk][nb][nb] Hermitian positive definite; Z: [nk][nb][m] -> C with C^H S C = 1."""
    L = np.linalg.cholesky(S)
    out = np.empty_like(Z)
    for k in range(S.shape[0]):
        Q, _ = np.linalg.qr(L[k].conj().T @ Z[k])
        out[k] = np.linalg.solve(L[k].conj().T, Q)
    return out


def load_problem(ctx, prob, iq_list=None):
    """Set basis and orthonormal states of a `synth.Problem` on a Context.
    Returns (C_k, C_kq[len(iq_list)]) as numpy arrays."""
    c, b = prob.cell, prob.basis
    ctx.set_basis(c.lattice, c.atoms, b.shell_atom, b.shell_l, b.shell_exp)
    iq_list = list(range(prob.nq)) if iq_list is None else list(iq_list)
    Ck = orthonormalise(ctx.overlap(prob.kpts), prob.Zk)
    Ckq = np.empty((len(iq_list), prob.nk, b.nbasis, prob.nc), np.complex128)
    for j, iq in enumerate(iq_list):
        Ckq[j] = orthonormalise(ctx.overlap(prob.kpts + prob.qpts[iq][None, :]), prob.zkq(iq))
    ctx.set_states(prob.kpts, Ck, prob.Ek, prob.qpts[iq_list], Ckq, prob.Ekq[iq_list])
    return Ck, Ckq


def load_optical(ctx, prob):
    """Basis and states of an optical-limit problem (a single q = 0): valence and
    conduction coefficients at the same k orthonormalised together, C = L^{-H} Q for
    [Z_v | Z_c] split by columns.  Returns (C_v, C_c)."""
    c, b = prob.cell, prob.basis
    ctx.set_basis(c.lattice, c.atoms, b.shell_atom, b.shell_l, b.shell_exp)
    C = orthonormalise(ctx.overlap(prob.kpts), np.concatenate([prob.Zk, prob.zkq(0)], axis=2))
    Cv, Cc = np.ascontiguousarray(C[:, :, :prob.nv]), np.ascontiguousarray(C[:, :, prob.nv:])
    ctx.set_states(prob.kpts, Cv, prob.Ek, prob.qpts[:1], Cc[None], prob.Ekq[:1])
    return Cv, Cc
