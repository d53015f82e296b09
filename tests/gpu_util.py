"""Shared set-up for the GPU parity tests."""
import numpy as np

from paper_2603_12326_gb300 import build, qcx


def context():
    build.build()
    return qcx.Context(0)


def set_oracle_states(ctx, p, iqs, Ck, Ckq):
    """Load basis and the oracle's orthonormal states for q indices iqs."""
    c, b = p.cell, p.basis
    ctx.set_basis(c.lattice, c.atoms, b.shell_atom, b.shell_l, b.shell_exp)
    ctx.set_states(p.kpts, Ck, p.Ek, p.qpts[iqs], np.stack(Ckq), p.Ekq[iqs])


def rel(a, b):
    """max |a - b| / max |b|."""
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / max(np.max(np.abs(b)), 1e-300))


def rel_spectrum(a, b, frac=1e-3):
    """Loss tables [nw][ng]: for every spectrum L(w) at fixed G, the largest
    relative error over the frequencies where L > frac * max_w L."""
    a = np.asarray(a)
    b = np.asarray(b)
    worst = 0.0
    for g in range(b.shape[1]):
        col = b[:, g]
        top = np.max(np.abs(col))
        if top <= 0:
            continue
        m = np.abs(col) > frac * top
        worst = max(worst, float(np.max(np.abs(a[m, g] - col[m]) / np.abs(col[m]))))
    return worst
