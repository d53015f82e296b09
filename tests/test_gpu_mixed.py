"""Mixed-precision GPU path (FP32 pair densities stored as three BF16 terms,
split-BF16 tcgen05 chi0 with FP32 accumulation, FP32 Gauss-Jordan inverse, the
FP64 diagonal correction for ill-conditioned blocks and the loss as a quadratic
form for the others) vs the FP64 CPU oracle.

Tolerances follow from the arithmetic: the contraction takes rho~ (the first two
BF16 terms of rho) on both sides, so its errors are W rho~'s three-term split
(2^-24 relative) and the one product left out (of that order), and chi0 carries
the FP32 rounding of its sums (5e-5 bound on its largest element); the inverse
amplifies eps errors by its condition number.  The loss functions must stay within 1e-4 relative wherever they
exceed 1e-3 of their per-q maximum (the bar the method is held to)."""
import numpy as np
import pytest

import synth
from oracle import rpa
from paper_2603_12326_gb300 import QCX_MIXED, qcx
from tests.gpu_util import context, rel, rel_spectrum, set_oracle_states

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = context()
    yield c
    c.close()


def _run(ctx, j, p, want_chi=True):
    rho = ctx.pair_density(j, p.G_int, QCX_MIXED, want=True)
    chi = ctx.chi0(j, p.w, p.eta, QCX_MIXED, want=want_chi)
    dinv, ed, resid = ctx.invert_eps(j, QCX_MIXED)
    L1, L2 = ctx.loss_function(j, QCX_MIXED)
    return rho, chi, dinv, ed, resid, L1, L2


def _check(o, rho, chi, dinv, ed, L1, L2):
    errs = {"rho": rel(rho, o["rho"]), "eps_diag": rel(ed, o["eps_diag"]),
            "eps_inv_diag": rel(dinv, o["eps_inv_diag"]),
            "L_lfe": rel_spectrum(L1, o["L_lfe"]), "L_nolfe": rel_spectrum(L2, o["L_nolfe"])}
    if chi is not None:
        errs["chi0"] = rel(chi, o["chi0"])
    print("mixed-path errors:", {k: f"{v:.2e}" for k, v in errs.items()})
    assert errs["rho"] < 5e-5
    assert errs.get("chi0", 0.0) < 5e-5
    assert errs["eps_diag"] < 5e-5
    assert errs["eps_inv_diag"] < 1e-4
    assert errs["L_lfe"] < 1e-4
    assert errs["L_nolfe"] < 1e-4


def test_small_workload_mixed(ctx):
    p = synth.make_small()
    iqs = [0, 4, 9]
    refs = []
    for iq in iqs:
        Ck, Ckq = rpa.states(p, iq)
        refs.append((Ck, Ckq, rpa.solve_q(p, iq, Ck, Ckq)))
    set_oracle_states(ctx, p, iqs, refs[0][0], [r[1] for r in refs])
    for j, (_, _, o) in enumerate(refs):
        rho, chi, dinv, ed, resid, L1, L2 = _run(ctx, j, p)
        _check(o, rho, chi, dinv, ed, L1, L2)


def test_ragged_mixed_single_chunk(ctx):
    """N_G = 13 (N tile 16, G' block partly empty), N_t = 120 (K padded to 256),
    7 frequencies (the last frequency pair has one empty accumulator)."""
    p = synth.make_tiny(shells_per_atom=3, n_k=2, nv=3, nc=5, ng=13, nq=1, nw=7)
    Ck, Ckq = rpa.states(p, 0)
    o = rpa.solve_q(p, 0, Ck, Ckq)
    set_oracle_states(ctx, p, [0], Ck, [Ckq])
    rho, chi, dinv, ed, resid, L1, L2 = _run(ctx, 0, p)
    _check(o, rho, chi, dinv, ed, L1, L2)


def test_split_g_range_mixed(ctx):
    """N_G = 229 > 192: the G axis is split into N chunks and the A-operand rows
    come from their own TMA tiles."""
    p = synth.make_tiny(shells_per_atom=3, n_k=2, nv=2, nc=6, ng=229, nq=1, nw=5)
    Ck, Ckq = rpa.states(p, 0)
    o = rpa.solve_q(p, 0, Ck, Ckq)
    set_oracle_states(ctx, p, [0], Ck, [Ckq])
    rho, chi, dinv, ed, resid, L1, L2 = _run(ctx, 0, p)
    _check(o, rho, chi, dinv, ed, L1, L2)


def test_fp64_correction_of_every_block(ctx):
    """Threshold 0: every block of a small-workload q goes through the FP64
    diagonal correction (the path the ill-conditioned blocks take); the result
    still matches the oracle and every block reports its correction."""
    p = synth.make_small()
    Ck, Ckq = rpa.states(p, 6)
    o = rpa.solve_q(p, 6, Ck, Ckq)
    set_oracle_states(ctx, p, [6], Ck, [Ckq])
    for bad in (-1.0, float("nan")):
        with pytest.raises(qcx.QcxError) as ei:
            ctx.set_refine_threshold(bad)
        assert ei.value.status == 1
    ctx.set_refine_threshold(0.0)
    try:
        rho, chi, dinv, ed, resid, L1, L2 = _run(ctx, 0, p)
    finally:
        ctx.set_refine_threshold(1.0e4)
    assert np.all(resid[1:] > 0.0) and np.all(resid < 1e-4)
    _check(o, rho, chi, dinv, ed, L1, L2)
    # the default threshold gives the same loss within the tolerance
    d2, _, r2 = ctx.invert_eps(0, QCX_MIXED)
    L1b, _ = ctx.loss_function(0, QCX_MIXED)
    assert rel_spectrum(L1b, o["L_lfe"]) < 1e-4


def test_mixed_recoil_spectrum_matches_oracle(ctx):
    """The rate end of the path in mixed precision: the loss tables of three
    small-workload q from the mixed path are binned over |q+G| on the GPU and fed
    to the FP64 rate (Eqs. (general_rate), (excitation_rate)); dR/dw and the
    recoil spectrum dR_Q are compared with the oracle's rate of the oracle's own
    loss tables, binned by the oracle, for both loss functions and both mediator
    limits.  Bar: 1e-4 relative where the value exceeds 1e-3 of its maximum."""
    from oracle import rate as orate
    p = synth.make_small(nq=3)
    iqs = [0, 1, 2]
    refs = []
    for iq in iqs:
        Ck, Ckq = rpa.states(p, iq)
        refs.append((Ck, Ckq, rpa.solve_q(p, iq, Ck, Ckq)))
    set_oracle_states(ctx, p, iqs, refs[0][0], [r[1] for r in refs])
    for j in range(3):
        _run(ctx, j, p, want_chi=False)
    edges = np.linspace(0.0, 2.5, 11)
    qmag = np.concatenate([np.linalg.norm(p.qpts[iq][None, :] + p.G_int @ p.cell.recip, axis=1) for iq in iqs])

    def masked(a, b):
        m = np.abs(b) > 1e-3 * np.max(np.abs(b))
        return float(np.max(np.abs(a[m] - b[m]) / np.abs(b[m])))

    worst = 0.0
    for which, key in ((0, "L_lfe"), (1, "L_nolfe")):
        Lb, cnt = ctx.bin_loss(iqs, which, edges, len(p.w))
        Lo, centres, co = orate.bin_loss(qmag, np.concatenate([r[2][key].T for r in refs], axis=0), edges)
        assert np.array_equal(cnt, co)
        nz = co > 0
        for params in (orate.HaloParams(), orate.HaloParams(m_med_eV=0.0, m_chi_eV=1e8)):
            dR, dQ = ctx.rate(centres[nz], p.w, Lb[nz], qcx.halo_params(**params.__dict__), nQ=12)
            dRo = orate.dR_dw(centres[nz], p.w, Lo[nz], params)
            dQo = orate.recoil_spectrum(p.w, dRo, params, 12)
            worst = max(worst, masked(dR, dRo), masked(dQ, dQo))
    print(f"mixed recoil spectrum vs oracle: {worst:.2e}")
    assert worst < 1e-4
