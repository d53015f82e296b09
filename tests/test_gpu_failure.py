"""The failure paths of the GPU path, made on purpose without faulting the GPU.

* A bounded wait that runs out: with the tensor-core kernel's copies withheld
  (a fault injected from the host, so nothing ever completes the stage
  barriers) and a short wait limit, every consumer's first wait gives up; the
  kernel stops its pipeline, lets its own copies and MMAs finish, frees its
  tensor memory and returns, and qcx_chi0 reports QCX_ERR_TIMEOUT.  The same
  context then computes the right answer.
* Argument checks of the two failure settings.

A singular dielectric matrix is exercised through the allocation-free entry
point (test_zz_no_alloc.py), which takes caller-built matrices: the per-q path
cannot form one, since for eta > 0 its eps has Im eps_GG > 0 at w > 0 and is
real with eps >= 1 at w = 0."""
import numpy as np
import pytest

import synth
from oracle import rpa
from paper_2603_12326_gb300 import QCX_MIXED, qcx
from tests.gpu_util import context, rel_spectrum, set_oracle_states

pytestmark = pytest.mark.gpu


def test_wait_timeout_is_reported_and_the_context_recovers():
    p = synth.make_small(nq=1, nw=12)
    Ck, Ckq = rpa.states(p, 0)
    o = rpa.solve_q(p, 0, Ck, Ckq)
    ctx = context()
    set_oracle_states(ctx, p, [0], Ck, [Ckq])
    ctx.pair_density(0, p.G_int, QCX_MIXED)
    ctx.set_wait_limit(200000)                  # ~0.1 ms of clock cycles
    ctx.set_fault_injection(True)
    for _ in range(2):
        with pytest.raises(qcx.QcxError) as e:
            ctx.chi0(0, p.w, p.eta, QCX_MIXED)
        assert e.value.status == 6              # QCX_ERR_TIMEOUT
        with pytest.raises(qcx.QcxError) as e:  # no eps was produced
            ctx.invert_eps(0, QCX_MIXED)
        assert e.value.status == 7
    ctx.set_fault_injection(False)
    ctx.set_wait_limit(4000000000)
    ctx.chi0(0, p.w, p.eta, QCX_MIXED)
    ctx.invert_eps(0, QCX_MIXED, want=False)
    L1, L2 = ctx.loss_function(0, QCX_MIXED)
    ctx.close()
    assert rel_spectrum(L1, o["L_lfe"]) < 1e-4 and rel_spectrum(L2, o["L_nolfe"]) < 1e-4


def test_failure_settings_reject_bad_arguments():
    ctx = context()
    for bad in (0, -5):
        with pytest.raises(qcx.QcxError) as e:
            ctx.set_wait_limit(bad)
        assert e.value.status == 1
    ctx.close()
    qcx.load()
    assert qcx.qcx_set_wait_limit(None, 100) == 1
    assert qcx.qcx_set_fault_injection(None, 1) == 1

