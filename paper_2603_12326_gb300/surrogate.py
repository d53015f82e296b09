"""Training data for the learned local-field correction.

Head loss functions of per-q solves (pair densities, chi0, inverse through
the library) are collected q chunk by q chunk, and turned into network inputs
and targets by qcx_surrogate_features.  This module only sequences C-ABI calls
and selects samples; it is input preparation, outside any timed region.
"""
from __future__ import annotations

import numpy as np

from . import QCX_MIXED
from .states import load_problem


def head_index(G_int) -> int:
    hits = np.nonzero(np.all(np.asarray(G_int) == 0, axis=1))[0]
    if len(hits) != 1:
        raise ValueError("the G list must contain G = 0 once")
    return int(hits[0])


def head_table(ctx, prob, iq_list, prec=QCX_MIXED, chunk=10):
    """L_LFE and L_noLFE heads [len(iq_list)][nw] of a `synth.Problem`."""
    iq_list = list(iq_list)
    h = head_index(prob.G_int)
    nw = len(prob.w)
    L1 = np.zeros((len(iq_list), nw))
    L2 = np.zeros((len(iq_list), nw))
    for c0 in range(0, len(iq_list), chunk):
        sel = iq_list[c0:c0 + chunk]
        load_problem(ctx, prob, sel)
        for j in range(len(sel)):
            ctx.pair_density(j, prob.G_int, prec)
            ctx.chi0(j, prob.w, prob.eta, prec)
            ctx.invert_eps(j, prec, want=False)
            a, b = ctx.loss_function(j, prec)
            L1[c0 + j] = a[:, h]
            L2[c0 + j] = b[:, h]
    return L1, L2


def keep_mask(L1, L2, drop=1e-3):
    """Samples whose L_LFE and L_noLFE both exceed `drop` of their spectrum's maximum."""
    return (L1 > drop * L1.max(axis=1, keepdims=True)) & (L2 > drop * L2.max(axis=1, keepdims=True))


def dataset(ctx, prob, iq_list, L1, L2, q_max, w_max, drop=1e-3):
    """(X [n][6], y [n], (q row, w index) of each kept sample) for q points
    iq_list of `prob` with head tables L1, L2 [len(iq_list)][nw]."""
    keep = keep_mask(L1, L2, drop)
    r, c = np.nonzero(keep)
    qv = prob.qpts[np.asarray(iq_list)[r]]
    X, y = ctx.surrogate_features(qv, prob.w[c], L2[r, c], q_max, w_max, L_lfe=L1[r, c])
    return X, y, (r, c)
