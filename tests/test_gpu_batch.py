"""Batched uneven instances (qcx_solve_batch) against the oracle.

The whole uneven workload (256 (q, w) instances over the small workload's
states, G sets {G : |q+G| < G_max} with N_G from 19 to 339) runs in one call,
the launch configuration the benchmark times; the oracle recomputes every
instance of two q points (including the largest, N_G = 339, and the
smallest, N_G = 19) one by one.  Tolerances: FP64 path 1e-10 relative, mixed
path 1e-4 relative, on the heads where the loss exceeds 1e-3 of the largest
compared head (absolute 1e-3 * tol * max below that)."""
import numpy as np
import pytest

import synth
from oracle import rpa
from paper_2603_12326_gb300 import QCX_FP64, QCX_MIXED, qcx
from tests.gpu_util import context

pytestmark = pytest.mark.gpu
SAMPLE_Q = (0, 8)


def _close(a, b, tol):
    a = np.asarray(a)
    b = np.asarray(b)
    top = np.max(np.abs(b))
    big = np.abs(b) > 1e-3 * top
    rel = np.max(np.abs(a[big] - b[big]) / np.abs(b[big]))
    small = np.max(np.abs(a[~big] - b[~big])) / top if np.any(~big) else 0.0
    return rel, small


@pytest.fixture(scope="module")
def uneven():
    p = synth.make_uneven()
    st = {iq: rpa.states(p, iq) for iq in range(p.nq)}
    e = p.extra
    sel = np.nonzero(np.isin(e["inst_q"], SAMPLE_Q))[0]
    L1, L2, ng = rpa.solve_instances(p, e["inst_q"][sel], e["inst_w"][sel], e["inst_gmax"][sel], st)
    assert e["inst_ng"][sel].max() == 339 and e["inst_ng"][sel].min() == 19
    return p, st, sel, L1, L2, ng


@pytest.fixture(scope="module")
def ctx(uneven):
    p, st, *_ = uneven
    c = context()
    b = p.basis
    c.set_basis(p.cell.lattice, p.cell.atoms, b.shell_atom, b.shell_l, b.shell_exp)
    Ck = st[0][0]
    c.set_states(p.kpts, Ck, p.Ek, p.qpts, np.stack([st[iq][1] for iq in range(p.nq)]), p.Ekq)
    yield c
    c.close()


@pytest.mark.parametrize("prec,tol", [(QCX_FP64, 1e-10), (QCX_MIXED, 1e-4)])
def test_uneven_batch_matches_oracle(ctx, uneven, prec, tol):
    p, st, sel, L1, L2, ngo = uneven
    e = p.extra
    a, b, ng = ctx.solve_batch(e["inst_q"], e["inst_w"], e["inst_gmax"], p.eta, prec)
    # G-set sizes of every instance, exactly
    assert np.array_equal(ng, e["inst_ng"])
    assert np.array_equal(ng[sel], ngo)
    r1, s1 = _close(a[sel], L1, tol)
    r2, s2 = _close(b[sel], L2, tol)
    print(f"prec {prec}: L_LFE rel {r1:.2e} (small {s1:.1e}), L_noLFE rel {r2:.2e} (small {s2:.1e})")
    assert r1 < tol and s1 < 1e-3 * tol
    assert r2 < tol and s2 < 1e-3 * tol
    info = ctx.batch_info()
    assert info["distinct_q"] == p.nq and info["max_ng"] == 339
    assert info["autotuned"] == (1 if prec == QCX_MIXED else 0)
    if prec == QCX_MIXED:
        # one tile-width cap per N_G class, each one of the widths the autotuner tries
        caps = (info["cap_ng65_128"], info["cap_ng129_192"], info["cap_ng193_up"])
        assert caps[0] in (64, 192) and caps[1] in (64, 128, 192) and caps[2] in (64, 128, 192), caps
        assert info["tile_cap"] == caps[2]


def test_mixed_batch_matches_fp64_batch_on_all_instances(ctx, uneven):
    p = uneven[0]
    e = p.extra
    a64, b64, _ = ctx.solve_batch(e["inst_q"], e["inst_w"], e["inst_gmax"], p.eta, QCX_FP64)
    a32, b32, _ = ctx.solve_batch(e["inst_q"], e["inst_w"], e["inst_gmax"], p.eta, QCX_MIXED)
    r1, s1 = _close(a32, a64, 1e-4)
    r2, s2 = _close(b32, b64, 1e-4)
    print(f"mixed vs FP64 over 256 instances: L_LFE {r1:.2e}, L_noLFE {r2:.2e}")
    assert r1 < 1e-4 and s1 < 1e-7 and r2 < 1e-4 and s2 < 1e-7


def test_graph_replay_is_deterministic_and_follows_new_frequencies(ctx, uneven):
    p = uneven[0]
    e = p.extra
    q, w, g = e["inst_q"], e["inst_w"], e["inst_gmax"]
    a1, b1, _ = ctx.solve_batch(q, w, g, p.eta, QCX_MIXED)
    info1 = ctx.batch_info()
    w2 = np.roll(w, 7)
    a2, b2, _ = ctx.solve_batch(q, w2, g, p.eta, QCX_MIXED)
    a3, b3, _ = ctx.solve_batch(q, w, g, p.eta, QCX_MIXED)
    assert ctx.batch_info() == info1            # same plan and graph
    assert np.array_equal(a1, a3) and np.array_equal(b1, b3)
    assert not np.array_equal(a1, a2)
    # the same instance list with rolled frequencies equals the FP64 path on those frequencies
    a64, _, _ = ctx.solve_batch(q, w2, g, p.eta, QCX_FP64)
    assert _close(a2, a64, 1e-4)[0] < 1e-4


def test_single_g_instances_and_edge_cases(ctx, uneven):
    p = uneven[0]
    c = p.cell
    qn = np.linalg.norm(p.qpts, axis=1)
    iq = np.arange(5, dtype=np.int32)      # |q| <= 0.95 (2 pi / a): no other G within 1.0001 |q|
    gmax = 1.0001 * qn[iq]                 # only G = 0 inside: N_G = 1
    w = p.w[5 + iq]
    for prec, tol in ((QCX_FP64, 1e-12), (QCX_MIXED, 1e-6)):
        a, b, ng = ctx.solve_batch(iq, w, gmax, p.eta, prec)
        assert np.all(ng == 1)
        assert np.max(np.abs(a - b) / np.abs(b)) < tol
    # G = 0 outside the cutoff, q index out of range, too many G vectors
    with pytest.raises(qcx.QcxError) as ei:
        ctx.solve_batch([0], [p.w[3]], [0.5 * qn[0]], p.eta, QCX_MIXED)
    assert ei.value.status == 1
    with pytest.raises(qcx.QcxError) as ei:
        ctx.solve_batch([p.nq], [p.w[3]], [3.0], p.eta, QCX_MIXED)
    assert ei.value.status == 1
    big = np.sqrt(80.0) * 2.0 * np.pi / c.a
    with pytest.raises(qcx.QcxError) as ei:
        ctx.solve_batch([0], [p.w[3]], [big], p.eta, QCX_FP64)
    assert ei.value.status == 8
