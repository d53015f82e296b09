"""Parity at the benchmark's full size: the first q of the mid workload
(512 k, N_b = 96, N_t = 65 536, N_G = 181, 200 w) through the mixed path in the
launch configuration bench.py times (one chi0 launch over all 200 w), and
through the FP64 path; the oracle recomputes four of the frequencies in full
(every G and G').  Tolerances as in the other parity tests: chi0 5e-5 and the
loss functions 1e-4 (per spectrum where L > 1e-3 of its maximum over the
sampled frequencies) for the mixed path, 1e-10 for the FP64 path."""
import numpy as np
import pytest

import synth
from oracle import rpa
from paper_2603_12326_gb300 import QCX_FP64, QCX_MIXED
from tests.gpu_util import context, rel, set_oracle_states

pytestmark = pytest.mark.gpu
SAMPLE_W = [40, 80, 120, 160]


@pytest.fixture(scope="module")
def mid():
    p = synth.make_mid(nq=1)
    Ck, Ckq = rpa.states(p, 0)
    o = rpa.solve_q(p, 0, Ck, Ckq, w=p.w[SAMPLE_W])
    return p, Ck, Ckq, o


def _masked(a, b, frac=1e-3):
    top = np.max(np.abs(b), axis=0, keepdims=True)
    m = np.abs(b) > frac * top
    return float(np.max(np.abs(a[m] - b[m]) / np.abs(b[m])))


def test_mid_workload_full_size_mixed(mid):
    p, Ck, Ckq, o = mid
    ctx = context()
    set_oracle_states(ctx, p, [0], Ck, [Ckq])
    ctx.pair_density(0, p.G_int, QCX_MIXED)
    chi = ctx.chi0(0, p.w, p.eta, QCX_MIXED, want=True)          # all 200 w in one launch
    ctx.invert_eps(0, QCX_MIXED, want=False)
    L1, L2 = ctx.loss_function(0, QCX_MIXED)
    ctx.close()
    e_chi = rel(chi[SAMPLE_W], o["chi0"])
    e1 = _masked(L1[SAMPLE_W], o["L_lfe"])
    e2 = _masked(L2[SAMPLE_W], o["L_nolfe"])
    print(f"mid full size, mixed: chi0 {e_chi:.2e}, L_LFE {e1:.2e}, L_noLFE {e2:.2e}")
    assert e_chi < 5e-5 and e1 < 1e-4 and e2 < 1e-4
    assert np.all(np.isfinite(L1)) and np.all(L1[1:] > -1e-8)     # the whole table: finite, no negative loss


def test_mid_workload_full_size_fp64(mid):
    p, Ck, Ckq, o = mid
    ctx = context()
    set_oracle_states(ctx, p, [0], Ck, [Ckq])
    ctx.pair_density(0, p.G_int, QCX_FP64)
    chi = ctx.chi0(0, p.w[SAMPLE_W], p.eta, QCX_FP64, want=True)
    ctx.invert_eps(0, QCX_FP64, want=False)
    L1, L2 = ctx.loss_function(0, QCX_FP64)
    ctx.close()
    assert rel(chi, o["chi0"]) < 1e-10
    assert rel(L1, o["L_lfe"]) < 1e-10 and rel(L2, o["L_nolfe"]) < 1e-10
