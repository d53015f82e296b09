"""CPU oracle for the all-electron RPA screening hot path (plain, slow, FP64).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the ``cpu_baseline`` / reference leg of ``bench.py`` may import this package.
The product path (``paper_2603_12326_gb300``) never imports it, and this
package never imports the product path: the two share no code.

Each function follows one step of the method as the paper states it:

* ``rpa.pair_ft`` / ``rpa.bloch_pair_table``: the matrix elements
  <i k| e^{-i(q+G).r} |j k'> of Eq. (RPA) for Bloch sums of Cartesian s/p
  Gaussians (Section III; Bloch form in Appendix C), written as the closed-form
  Gaussian-product integral summed over lattice translations.
* ``rpa.pair_density``: rho_vck(q+G) = <c,k+q| e^{i(q+G).r} |v,k>.
* ``rpa.transition_weights``: the retarded energy denominators of Eq. (RPA)
  for the T=0 occupations (f = 2 valence, 0 conduction).
* ``rpa.chi0`` / ``rpa.dielectric_matrix``: Eq. (RPA).
* ``rpa.loss_functions``: Eq. (eps_LFE), Eq. (eps_noLFE) and the loss
  function Im[-1/eps] of Eq. (dynamic_structure_factor).
* ``rate``: Eqs. (general_rate), (cross_section), (F_DM_limits),
  (excitation_rate) in the nonrelativistic halo limit of Appendix A.
* ``mlp``: the learned local-field correction (no counterpart in the paper):
  network, Gaussian negative log-likelihood, back-propagation and Adam.
* ``spectral``: the spectral route to chi0 (Eq. (eRPA_spectral) binned on an
  energy grid once per q, the principal part by the Kramers-Kronig step with
  the direct sum's broadening); no GPU path yet.

Parity status of every function is listed in the module docstrings; each is
pinned by a test in ``tests/test_oracle_*.py``.
"""
