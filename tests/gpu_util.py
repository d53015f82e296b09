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


def rel_masked(a, b, frac=1e-3):
    """max relative error over entries with |b| > frac * max |b| (per leading index)."""
    a = np.asarray(a)
    b = np.asarray(b)
    worst = 0.0
    for i in range(b.shape[0]):
        m = np.abs(b[i]) > frac * np.max(np.abs(b[i]))
        if m.any():
            worst = max(worst, float(np.max(np.abs(a[i][m] - b[i][m]) / np.abs(b[i][m]))))
    return worst
