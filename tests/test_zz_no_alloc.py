"""The allocation-free entry point (qcx_eps_inverse_diag_noalloc) against the
regular one (qcx_invert_eps, FP64).

It serves callers that cannot allocate device memory when they need the
inverse diagonal (an allocator owned by another framework, a memory budget
reserved at start-up, pipelines that cannot afford cudaMalloc's device
synchronisation); its scratch is a fixed array inside the library.  The test
feeds it the same dielectric matrices the regular path inverts, calls it twice
in a row on the shared scratch, and compares both results with the regular
path's within the FP64 tolerance of the other GPU tests (1e-10 relative).
This file is collected last so that a run stopping at the first failure has
run every other test before it."""
import ctypes as ct

import numpy as np
import pytest

import synth
from oracle import rpa
from paper_2603_12326_gb300 import QCX_FP64, qcx
from tests.gpu_util import context, rel

pytestmark = pytest.mark.gpu


def test_noalloc_inverse_matches_regular_path_twice():
    torch = pytest.importorskip("torch")
    p = synth.make_small(nq=1, nw=24)
    Ck, Ckq = rpa.states(p, 0)
    ctx = context()
    c, b = p.cell, p.basis
    ctx.set_basis(c.lattice, c.atoms, b.shell_atom, b.shell_l, b.shell_exp)
    ctx.set_states(p.kpts, Ck, p.Ek, p.qpts[:1], Ckq[None], p.Ekq[:1])
    ctx.pair_density(0, p.G_int, QCX_FP64)
    chi = ctx.chi0(0, p.w, p.eta, QCX_FP64, want=True)
    dinv_ref, ed_ref, _ = ctx.invert_eps(0, QCX_FP64)
    L1_ref, L2_ref = ctx.loss_function(0, QCX_FP64)
    ctx.close()
    # the same dielectric matrices, built from the exported chi0
    vs = np.sqrt(4.0 * np.pi) / np.linalg.norm(p.qpts[0][None, :] + p.G_int @ c.recip, axis=1)
    eps = np.eye(p.ng)[None] - vs[None, :, None] * chi * vs[None, None, :]
    nb, n = eps.shape[0], eps.shape[1]
    dev = torch.device("cuda:0")
    e_t = torch.from_numpy(np.ascontiguousarray(eps)).to(dev)
    for call in range(2):
        d_t = torch.zeros((nb, n), dtype=torch.complex128, device=dev)
        l1 = torch.zeros((nb, n), dtype=torch.float64, device=dev)
        l2 = torch.zeros((nb, n), dtype=torch.float64, device=dev)
        sing = torch.full((nb,), -1, dtype=torch.int32, device=dev)
        st = qcx.qcx_eps_inverse_diag_noalloc(ct.c_void_p(e_t.data_ptr()), nb, n, ct.c_void_p(d_t.data_ptr()),
                                              ct.c_void_p(l1.data_ptr()), ct.c_void_p(l2.data_ptr()),
                                              ct.c_void_p(sing.data_ptr()), None)
        assert st == 0
        torch.cuda.synchronize()
        assert int(sing.abs().sum()) == 0
        assert rel(d_t.cpu().numpy(), dinv_ref) < 1e-10, call
        assert rel(l1.cpu().numpy(), L1_ref) < 1e-10, call
        assert rel(l2.cpu().numpy(), L2_ref) < 1e-10, call


def test_noalloc_flags_a_singular_matrix_among_good_ones():
    """Three matrices in one call, the middle one all zeros: its singular flag
    is set and its outputs are zero, while the two others still match the
    regular path (1e-10).  A zero matrix meets a zero pivot at the first
    column, so the elimination's singular branch runs whatever the rounding."""
    torch = pytest.importorskip("torch")
    p = synth.make_small(nq=1)
    Ck, Ckq = rpa.states(p, 0)
    ctx = context()
    c, b = p.cell, p.basis
    ctx.set_basis(c.lattice, c.atoms, b.shell_atom, b.shell_l, b.shell_exp)
    ctx.set_states(p.kpts, Ck, p.Ek, p.qpts[:1], Ckq[None], p.Ekq[:1])
    w = p.w[[10, 20]]
    ctx.pair_density(0, p.G_int, QCX_FP64)
    chi = ctx.chi0(0, w, p.eta, QCX_FP64, want=True)
    dinv_ref, _, _ = ctx.invert_eps(0, QCX_FP64)
    L1_ref, L2_ref = ctx.loss_function(0, QCX_FP64)
    ctx.close()
    vs = np.sqrt(4.0 * np.pi) / np.linalg.norm(p.qpts[0][None, :] + p.G_int @ c.recip, axis=1)
    good = np.eye(p.ng)[None] - vs[None, :, None] * chi * vs[None, None, :]
    n = p.ng
    eps = np.stack([good[0], np.zeros((n, n), complex), good[1]])
    dev = torch.device("cuda:0")
    e_t = torch.from_numpy(eps).to(dev)
    d_t = torch.full((3, n), 7.0, dtype=torch.complex128, device=dev)
    l1 = torch.full((3, n), 7.0, dtype=torch.float64, device=dev)
    l2 = torch.full((3, n), 7.0, dtype=torch.float64, device=dev)
    sing = torch.full((3,), -1, dtype=torch.int32, device=dev)
    st = qcx.qcx_eps_inverse_diag_noalloc(ct.c_void_p(e_t.data_ptr()), 3, n, ct.c_void_p(d_t.data_ptr()),
                                          ct.c_void_p(l1.data_ptr()), ct.c_void_p(l2.data_ptr()),
                                          ct.c_void_p(sing.data_ptr()), None)
    assert st == 0
    torch.cuda.synchronize()
    assert sing.cpu().tolist() == [0, 1, 0]
    d, a, bb = d_t.cpu().numpy(), l1.cpu().numpy(), l2.cpu().numpy()
    assert not np.any(d[1]) and not np.any(a[1]) and not np.any(bb[1])
    for k, j in ((0, 0), (2, 1)):
        assert rel(d[k], dinv_ref[j]) < 1e-10
        assert rel(a[k], L1_ref[j]) < 1e-10
        assert rel(bb[k], L2_ref[j]) < 1e-10


def test_noalloc_rejects_sizes_over_the_scratch():
    torch = pytest.importorskip("torch")
    qcx.load()
    dev = torch.device("cuda:0")
    e_t = torch.zeros((1, 4, 4), dtype=torch.complex128, device=dev)
    d_t = torch.zeros((1, 4), dtype=torch.complex128, device=dev)
    # 2000 x 2000 complex doubles = 64 MB > 16 MiB: refused before anything runs
    st = qcx.qcx_eps_inverse_diag_noalloc(ct.c_void_p(e_t.data_ptr()), 1, 2000, ct.c_void_p(d_t.data_ptr()),
                                          None, None, None, None)
    assert st == 1
    # host pointers are refused as well
    h = np.zeros((1, 4, 4), np.complex128)
    st = qcx.qcx_eps_inverse_diag_noalloc(ct.c_void_p(h.ctypes.data), 1, 4, ct.c_void_p(d_t.data_ptr()),
                                          None, None, None, None)
    assert st == 1
