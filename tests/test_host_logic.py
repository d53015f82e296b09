"""Host-side selection logic of the learned correction's training data (CPU):
the head (G = 0) lookup and the drop rule — a (q, w) sample is kept only when
both its L_LFE and its L_noLFE exceed 1e-3 of the maximum of their own
spectrum (so w = 0, where the loss vanishes, is always dropped)."""
import numpy as np
import pytest

from paper_2603_12326_gb300 import surrogate


def test_head_index_finds_g_zero_once():
    G = np.array([[1, 0, 0], [0, 0, 0], [0, -1, 1]])
    assert surrogate.head_index(G) == 1
    with pytest.raises(ValueError):
        surrogate.head_index(G[[0, 2]])                  # no G = 0
    with pytest.raises(ValueError):
        surrogate.head_index(G[[1, 0, 1]])               # G = 0 twice


def test_keep_mask_is_per_spectrum_and_needs_both_losses():
    w = np.linspace(0.0, 1.0, 6)
    L1 = np.array([np.sin(np.pi * w) * 10.0,             # spectrum maximum 10
                   np.sin(np.pi * w) * 1e-6])            # tiny spectrum: compared with its own maximum
    L2 = L1.copy()
    L2[0, 2] = 5e-3 * L2[0].max() * 0.1                  # L_noLFE under the bar at one frequency only
    keep = surrogate.keep_mask(L1, L2)
    assert not keep[:, 0].any() and not keep[:, -1].any()    # sin(0) = sin(pi) ~ 0: the loss vanishes
    assert keep[1, 1:5].all()                            # the scale of a spectrum does not matter
    assert not keep[0, 2] and keep[0, 1] and keep[0, 3]  # one loss under its bar drops the sample
    # exactly at the bar is dropped, just above is kept
    a = np.array([[1.0, 1e-3, 1.0001e-3]])
    assert surrogate.keep_mask(a, a).tolist() == [[True, False, True]]
