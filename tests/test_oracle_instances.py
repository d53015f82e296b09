"""Pins of the oracle's uneven-instance solver (one (q, w) block per instance,
G set {G : |q+G| < G_max}, head of the loss functions).

References: the shell counts of the body-centred-cubic reciprocal lattice of
the FCC cell (a fact of the lattice, not of the code), the N_G = 1 limit in
which local fields cannot act (Eq. (eps_LFE) equals Eq. (eps_noLFE)), the
single-oscillator closed form of that limit, and the per-q path (`solve_q`,
pinned elsewhere) run on the same G set listed in a shuffled order."""
import numpy as np
import pytest

import synth
from oracle import rpa


def test_g_ball_counts_match_bcc_shell_closures():
    """|G|^2 (2 pi / a)^-2 <= 4, 8, 32, 48, 59 hold 15, 27, 181, 339, 531
    reciprocal vectors of the FCC cell (catches a wrong bounding box, a
    transposed reciprocal basis or a <= / < slip at the cutoff)."""
    c = synth.diamond_cell()
    unit = 2.0 * np.pi / c.a
    for r2, n in [(4, 15), (8, 27), (32, 181), (48, 339), (59, 531)]:
        assert rpa.g_ball(c.recip, np.zeros(3), np.sqrt(r2 + 0.5) * unit).shape[0] == n
        # the shell itself lies on the cutoff: strictly-below excludes it
        assert rpa.g_ball(c.recip, np.zeros(3), np.sqrt(r2) * unit * (1 - 1e-12)).shape[0] < n


def test_g_ball_shifted_by_q_is_the_ball_around_minus_q():
    """{G : |q+G| < g} for q = a reciprocal vector G0 is {G - G0 : |G| < g}."""
    c = synth.diamond_cell()
    G0 = np.array([1, -1, 2])
    q = G0 @ c.recip
    g = np.sqrt(8.5) * 2.0 * np.pi / c.a
    a = {tuple(x) for x in rpa.g_ball(c.recip, q, g)}
    b = {tuple(x - G0) for x in rpa.g_ball(c.recip, np.zeros(3), g)}
    assert a == b and len(a) == 27


@pytest.fixture(scope="module")
def tiny():
    p = synth.make_tiny(seed=11, shells_per_atom=2, n_k=2, nv=2, nc=3, ng=9, nq=2, nw=8)
    return p, {iq: rpa.states(p, iq) for iq in range(p.nq)}


def test_single_g_instance_has_no_local_fields(tiny):
    """With only G = 0 inside the cutoff, L_LFE = L_noLFE exactly, and both
    equal the single-oscillator form -Im 1/eps with
    eps = 1 - (4 pi/|q|^2) (2/(N_k V)) sum_t W_t |rho_t(0)|^2."""
    p, st = tiny
    c = p.cell
    iq = 0
    q = p.qpts[iq]
    gmax = 1.0001 * np.linalg.norm(q)
    assert rpa.g_ball(c.recip, q, gmax).shape[0] == 1
    w = p.w[3]
    L1, L2, ng = rpa.solve_instances(p, [iq], [w], [gmax], st)
    assert ng[0] == 1
    assert L1[0] == pytest.approx(L2[0], rel=1e-13, abs=0)
    Ck, Ckq = st[iq]
    b = p.basis
    rho0 = rpa.pair_density_lean(c.lattice, c.atoms, b.shell_atom, b.shell_l, b.shell_exp, p.kpts,
                                 q[None, :], Ck, Ckq)[:, 0]
    dE = (p.Ekq[iq][:, None, :] - p.Ek[:, :, None]).reshape(-1)
    Wt = 2.0 * dE / ((w + 1j * p.eta) ** 2 - dE ** 2)
    eps = 1.0 - 4.0 * np.pi / np.dot(q, q) * 2.0 / (p.nk * c.volume) * np.sum(Wt * np.abs(rho0) ** 2)
    assert L1[0] == pytest.approx(-(1.0 / eps).imag, rel=1e-12)


def test_instances_match_per_q_path_on_shuffled_g_list(tiny):
    """Each instance equals `solve_q` run on the same G set in a shuffled
    order at the instance's frequency, read at G = 0 (catches a wrong head
    index, columns of the wrong G taken from the union, or a q mix-up between
    instances)."""
    p, st = tiny
    c = p.cell
    unit = 2.0 * np.pi / c.a
    rng = np.random.default_rng(5)
    inst_q = [0, 1, 0, 1, 0]
    inst_w = [p.w[2], p.w[5], p.w[7], p.w[1], p.w[4]]
    inst_g = [3.1 * unit, 2.9 * unit, 3.6 * unit, 3.4 * unit, 3.3 * unit]
    L1, L2, ng = rpa.solve_instances(p, inst_q, inst_w, inst_g, st)
    for i in range(len(inst_q)):
        G = rpa.g_ball(c.recip, p.qpts[inst_q[i]], inst_g[i])
        G = G[rng.permutation(G.shape[0])]
        pi = synth.truncate(synth.make_tiny(seed=11, shells_per_atom=2, n_k=2, nv=2, nc=3, ng=9, nq=2, nw=8),
                            None, None)
        pi.G_int = G
        Ck, Ckq = st[inst_q[i]]
        o = rpa.solve_q(pi, inst_q[i], Ck, Ckq, w=[inst_w[i]])
        h = int(np.nonzero(np.all(G == 0, axis=1))[0][0])
        assert ng[i] == G.shape[0] > 9
        assert L1[i] == pytest.approx(o["L_lfe"][0, h], rel=1e-12)
        assert L2[i] == pytest.approx(o["L_nolfe"][0, h], rel=1e-12)
    # local fields change the head once more than one G is kept
    assert np.max(np.abs(L1 - L2) / np.abs(L2)) > 1e-3
