"""The optical limit q -> 0 (Appendix C) on the GPU against its oracle
(oracle/optical.py): the pair densities with the G = 0 row replaced by
-i qhat.<c k|grad|v k>/dE (the other rows at q = 0), chi0 of the head, wings and
body, the inverse and both loss functions; FP64 at 1e-10 relative to the
largest value, the mixed path at its bars (chi0 5e-5, loss 1e-4 per spectrum
where L > 1e-3 of its maximum).  The direction is passed unnormalised."""
import numpy as np
import pytest

import synth
from oracle import optical
from paper_2603_12326_gb300 import QCX_FP64, QCX_MIXED, qcx
from tests.gpu_util import context, rel, rel_spectrum

pytestmark = pytest.mark.gpu
QHAT = np.array([1.0, 0.4, -0.3])


@pytest.fixture(scope="module")
def opt():
    p = synth.make_optical("small", nw=24)
    Cv, Cc = optical.states_joint(p)
    return p, Cv, Cc, optical.solve_optical(p, QHAT, Cv, Cc)


def _ctx(p, Cv, Cc):
    ctx = context()
    c, b = p.cell, p.basis
    ctx.set_basis(c.lattice, c.atoms, b.shell_atom, b.shell_l, b.shell_exp)
    ctx.set_states(p.kpts, Cv, p.Ek, p.qpts[:1], Cc[None], p.Ekq[:1])
    return ctx


def test_optical_limit_fp64_matches_oracle(opt):
    p, Cv, Cc, o = opt
    ctx = _ctx(p, Cv, Cc)
    rho = ctx.pair_density_optical(0, p.G_int, 2.5 * QHAT, QCX_FP64, want=True)
    chi = ctx.chi0(0, p.w, p.eta, QCX_FP64, want=True)
    d, e, _ = ctx.invert_eps(0, QCX_FP64)
    L1, L2 = ctx.loss_function(0, QCX_FP64)
    ctx.close()
    g0 = o["g0"]
    assert rel(rho[:, g0], o["rho"][:, g0]) < 1e-10          # the optical column alone
    assert rel(rho, o["rho"]) < 1e-10
    assert rel(chi, o["chi0"]) < 1e-10
    assert rel(d, o["eps_inv_diag"]) < 1e-10 and rel(e, o["eps_diag"]) < 1e-10
    assert rel(L1, o["L_lfe"]) < 1e-10 and rel(L2, o["L_nolfe"]) < 1e-10


def test_optical_limit_mixed_at_the_mixed_bar(opt):
    p, Cv, Cc, o = opt
    ctx = _ctx(p, Cv, Cc)
    ctx.pair_density_optical(0, p.G_int, QHAT, QCX_MIXED)
    chi = ctx.chi0(0, p.w, p.eta, QCX_MIXED, want=True)
    ctx.invert_eps(0, QCX_MIXED, want=False)
    L1, L2 = ctx.loss_function(0, QCX_MIXED)
    ctx.close()
    e = rel(chi, o["chi0"]), rel_spectrum(L1, o["L_lfe"]), rel_spectrum(L2, o["L_nolfe"])
    print("optical limit, mixed vs oracle: chi0 %.2e, L_LFE %.2e, L_noLFE %.2e" % e)
    assert e[0] < 5e-5 and e[1] < 1e-4 and e[2] < 1e-4


def test_optical_limit_arguments_are_checked(opt):
    p, Cv, Cc, o = opt
    ctx = _ctx(p, Cv, Cc)
    no_g0 = p.G_int[np.any(p.G_int != 0, axis=1)]
    for args in ((0, no_g0, QHAT), (0, p.G_int, np.zeros(3)), (0, np.vstack([p.G_int, p.G_int[:1]]), QHAT)):
        with pytest.raises(qcx.QcxError) as e:
            ctx.pair_density_optical(*args, QCX_FP64)
        assert e.value.status == 1
    ctx.close()
    # a q that is not zero
    q = synth.make_small(nq=1, nw=4)
    from oracle import rpa
    Ck, Ckq = rpa.states(q, 0)
    ctx = context()
    c, b = q.cell, q.basis
    ctx.set_basis(c.lattice, c.atoms, b.shell_atom, b.shell_l, b.shell_exp)
    ctx.set_states(q.kpts, Ck, q.Ek, q.qpts[:1], Ckq[None], q.Ekq[:1])
    with pytest.raises(qcx.QcxError) as e:
        ctx.pair_density_optical(0, q.G_int, QHAT, QCX_FP64)
    assert e.value.status == 1
    ctx.close()
