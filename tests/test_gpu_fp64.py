"""Plain FP64 GPU path vs the CPU oracle (elementwise, <= 1e-10 relative).

Tolerance: the two sides evaluate the same sums in different orders and
truncate the lattice sum differently below e^-46 (box vs sphere), so the
differences are rounding-level; 1e-10 of the largest magnitude per array is
the bar."""
import numpy as np
import pytest

import synth
from oracle import rate as orate
from oracle import rpa
from paper_2603_12326_gb300 import QCX_FP64, qcx
from tests.gpu_util import context, rel, set_oracle_states

pytestmark = pytest.mark.gpu
TOL = 1e-10


@pytest.fixture(scope="module")
def ctx():
    c = context()
    yield c
    c.close()


def _oracle_q(p, iq):
    Ck, Ckq = rpa.states(p, iq)
    return Ck, Ckq, rpa.solve_q(p, iq, Ck, Ckq)


def _gpu_q(ctx, j, p, prec=QCX_FP64):
    rho = ctx.pair_density(j, p.G_int, prec, want=True)
    chi = ctx.chi0(j, p.w, p.eta, prec, want=True)
    dinv, ed, resid = ctx.invert_eps(j, prec)
    L1, L2 = ctx.loss_function(j, prec)
    return rho, chi, dinv, ed, L1, L2


def test_overlap_matches_oracle(ctx):
    p = synth.make_small(nq=1)
    c, b = p.cell, p.basis
    ctx.set_basis(c.lattice, c.atoms, b.shell_atom, b.shell_l, b.shell_exp)
    k = np.vstack([p.kpts[:6], [[0.13, -0.21, 0.05]]])
    S = ctx.overlap(k)
    So = rpa.overlap(c.lattice, c.atoms, b.shell_atom, b.shell_l, b.shell_exp, k)
    assert rel(S, So) < 1e-12


@pytest.mark.parametrize("iqs", [[0, 4, 9]])
def test_small_workload_fp64(ctx, iqs):
    p = synth.make_small()
    ref = [_oracle_q(p, iq) for iq in iqs]
    set_oracle_states(ctx, p, iqs, ref[0][0], [r[1] for r in ref])
    for j, (_, _, o) in enumerate(ref):
        rho, chi, dinv, ed, L1, L2 = _gpu_q(ctx, j, p)
        assert rel(rho, o["rho"]) < TOL
        assert rel(chi, o["chi0"]) < TOL
        assert rel(ed, o["eps_diag"]) < TOL
        assert rel(dinv, o["eps_inv_diag"]) < TOL
        assert rel(L1, o["L_lfe"]) < TOL
        assert rel(L2, o["L_nolfe"]) < TOL


def test_ragged_sizes_fp64(ctx):
    """N_G = 13 (not a tile multiple), N_t = 8*3*5 = 120 (not a multiple of the
    16-transition stage), 7 frequencies (not a multiple of 4)."""
    p = synth.make_tiny(shells_per_atom=3, n_k=2, nv=3, nc=5, ng=13, nq=2, nw=7)
    ref = [_oracle_q(p, iq) for iq in (0, 1)]
    set_oracle_states(ctx, p, [0, 1], ref[0][0], [r[1] for r in ref])
    for j, (_, _, o) in enumerate(ref):
        rho, chi, dinv, ed, L1, L2 = _gpu_q(ctx, j, p)
        assert rel(rho, o["rho"]) < TOL
        assert rel(chi, o["chi0"]) < TOL
        assert rel(dinv, o["eps_inv_diag"]) < TOL
        assert rel(L1, o["L_lfe"]) < TOL
        assert rel(L2, o["L_nolfe"]) < TOL


def test_single_g_identity(ctx):
    """N_G = 1: the loss with and without local fields coincide (Eq. (eps_LFE) vs (eps_noLFE))."""
    p = synth.make_small(nq=1, nw=50)
    p.G_int = p.G_int[:1]
    Ck, Ckq = rpa.states(p, 0)
    set_oracle_states(ctx, p, [0], Ck, [Ckq])
    *_, L1, L2 = _gpu_q(ctx, 0, p)
    assert np.max(np.abs(L1 - L2)) <= 1e-14 * np.max(np.abs(L1))


def test_binning_and_rate_match_oracle(ctx):
    p = synth.make_small(nq=3)
    iqs = [0, 1, 2]
    ref = [_oracle_q(p, iq) for iq in iqs]
    set_oracle_states(ctx, p, iqs, ref[0][0], [r[1] for r in ref])
    for j in range(3):
        _gpu_q(ctx, j, p)
    edges = np.linspace(0.0, 2.5, 11)
    for which, key in ((0, "L_lfe"), (1, "L_nolfe")):
        Lb, cnt = ctx.bin_loss(iqs, which, edges, len(p.w))
        qmag = np.concatenate([np.linalg.norm(p.qpts[iq][None, :] + p.G_int @ p.cell.recip, axis=1) for iq in iqs])
        Lall = np.concatenate([r[2][key].T for r in ref], axis=0)   # [(q,G)][w]
        Lo, centres, co = orate.bin_loss(qmag, Lall, edges)
        assert np.array_equal(cnt, co)
        assert rel(Lb, Lo) < TOL
    nz = cnt > 0
    qb = centres[nz]
    Lq = Lb[nz]
    for params in (orate.HaloParams(), orate.HaloParams(m_med_eV=0.0, m_chi_eV=1e8)):
        hp = qcx.halo_params(**params.__dict__)
        dR, dQ = ctx.rate(qb, p.w, Lq, hp, nQ=12)
        dRo = orate.dR_dw(qb, p.w, Lq, params)
        dQo = orate.recoil_spectrum(p.w, dRo, params, 12)
        assert rel(dR, dRo) < 1e-12
        assert rel(dQ, dQo) < 1e-12


def test_call_order_and_argument_errors(ctx):
    p = synth.make_tiny(nq=1)
    Ck, Ckq = rpa.states(p, 0)
    set_oracle_states(ctx, p, [0], Ck, [Ckq])
    with pytest.raises(qcx.QcxError) as e:
        ctx.chi0(0, p.w, p.eta, QCX_FP64)
    assert e.value.status == 7                       # no pair densities yet
    with pytest.raises(qcx.QcxError) as e:
        ctx.pair_density(5, p.G_int, QCX_FP64)      # q out of range
    assert e.value.status == 1
    ctx.pair_density(0, p.G_int, QCX_FP64)
    with pytest.raises(qcx.QcxError) as e:
        ctx.chi0(0, p.w, -1.0, QCX_FP64)             # eta <= 0
    assert e.value.status == 1
    with pytest.raises(qcx.QcxError) as e:
        ctx.chi0(0, np.array([0.1, np.nan]), 0.01, QCX_FP64)
    assert e.value.status == 1
    with pytest.raises(qcx.QcxError) as e:
        ctx.loss_function(0, QCX_FP64)               # not inverted yet
    assert e.value.status == 7
    # the context is still usable after the failures
    ctx.chi0(0, p.w, p.eta, QCX_FP64)
    ctx.invert_eps(0, QCX_FP64)
    L1, L2 = ctx.loss_function(0, QCX_FP64)
    assert np.all(np.isfinite(L1))


def test_loss_tables_follow_the_computation(ctx):
    """The loss tables of a q are readable only after qcx_invert_eps on the
    current pair densities, chi0 and states; recomputing any of them resets the
    tables of that q (their device buffers are kept and reused).  Empty G and
    frequency lists are argument errors."""
    p = synth.make_tiny(seed=5, nq=2, nw=6)
    st = [rpa.states(p, iq) for iq in range(2)]
    set_oracle_states(ctx, p, [0, 1], st[0][0], [s[1] for s in st])
    edges = np.linspace(0.0, 10.0, 11)
    for iq in range(2):
        ctx.pair_density(iq, p.G_int, QCX_FP64)
        ctx.chi0(iq, p.w, p.eta, QCX_FP64)
        ctx.invert_eps(iq, QCX_FP64)
    L0, _ = ctx.loss_function(0, QCX_FP64)
    ctx.bin_loss([0, 1], 0, edges, len(p.w))

    def stale(iq):
        with pytest.raises(qcx.QcxError) as e:
            ctx.loss_function(iq, QCX_FP64)
        assert e.value.status == 7

    ctx.pair_density(0, p.G_int, QCX_FP64)           # new pair densities of q 0
    stale(0)
    ctx.loss_function(1, QCX_FP64)                   # q 1 untouched
    with pytest.raises(qcx.QcxError) as e:
        ctx.bin_loss([0, 1], 0, edges, len(p.w))
    assert e.value.status == 7
    ctx.chi0(0, p.w, p.eta, QCX_FP64)
    stale(0)
    ctx.invert_eps(0, QCX_FP64)
    La, _ = ctx.loss_function(0, QCX_FP64)
    assert np.allclose(La, L0, rtol=1e-14, atol=0)   # same inputs, same tables
    ctx.chi0(0, p.w[:3], p.eta, QCX_FP64)            # other frequencies
    stale(0)
    ctx.invert_eps(0, QCX_FP64)
    Lb, _ = ctx.loss_function(0, QCX_FP64)
    assert Lb.shape == (3, p.G_int.shape[0]) and np.allclose(Lb, L0[:3], rtol=1e-12, atol=0)
    set_oracle_states(ctx, p, [0, 1], st[0][0], [s[1] for s in st])   # new states: every table resets
    stale(0)
    stale(1)
    with pytest.raises(qcx.QcxError) as e:
        ctx.pair_density(0, p.G_int[:0], QCX_FP64)   # no G vectors
    assert e.value.status == 1
    ctx.pair_density(0, p.G_int, QCX_FP64)
    with pytest.raises(qcx.QcxError) as e:
        ctx.chi0(0, np.zeros(0), p.eta, QCX_FP64)    # no frequencies
    assert e.value.status == 1
