/*
 * qcx.h -- C ABI of libqcx, a GB300 (sm_103a) implementation of the
 * data-parallel hot path of all-electron RPA screening with local-field
 * effects (arXiv 2603.12326, "QCDark2").
 *
 * The path, in the paper's order:
 *   pair densities  rho_vck(q+G) = <c,k+q| e^{i(q+G).r} |v,k>      (Eq. (RPA) numerator, Sec. II.D, III)
 *   chi0_GG'(q,w)   = 2/(N_k V) sum_t W_t(w) rho_t(G)^* rho_t(G')   (Eq. (RPA))
 *   eps_GG'         = delta_GG' - v^1/2(q+G) chi0_GG' v^1/2(q+G')    (Eq. (RPA))
 *   [eps^-1]_GG     -> eps(w, q+G) = 1/[eps^-1]_GG                   (Eq. (eps_LFE))
 *   eps_GG          -> eps^noLFE(w, q+G)                             (Eq. (eps_noLFE))
 *   L = Im[-1/eps]  and the halo scattering rate / recoil spectrum  (Eqs. (dynamic_structure_factor),
 *                                                                      (cross_section), (excitation_rate))
 * with W_t(w) = 1/(w - dE_t + i eta) - 1/(w + dE_t + i eta) (T = 0 occupations,
 * retarded broadening) and v^1/2(k) = sqrt(4 pi)/|k|.
 *
 * Units: Hartree atomic units (bohr, Hartree) at every entry point except
 * qcx_halo_params, which uses the units named in its fields.
 *
 * Conventions for every entry point
 *  - Inputs are copied before the call returns; the caller keeps ownership.
 *  - Array arguments may be host or device pointers; residency is detected
 *    with cudaPointerGetAttributes.  Device pointers must belong to the
 *    context's device.
 *  - Outputs are caller-owned.  A NULL output pointer means "not wanted".
 *    When every output of a call is in device memory the call is
 *    asynchronous on the context's stream; a host output makes the call
 *    synchronise before returning.
 *  - Complex numbers are qcx_c64 {re, im} (two doubles, interleaved).
 *  - Errors: every call returns a qcx_status; on failure the context keeps
 *    a message (qcx_last_error) and stays usable.  No C++ exception crosses
 *    the ABI.  Calls made out of order return QCX_ERR_STATE.
 *  - One context is used by one host thread at a time.
 *  - Index t of a transition is (k * n_v + v) * n_c + c.
 *  - G vectors are integer coefficients on the reciprocal basis b_1, b_2,
 *    b_3 (a_i . b_j = 2 pi delta_ij).
 */
#ifndef QCX_H
#define QCX_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct qcx_ctx qcx_ctx;

typedef enum {
    QCX_OK = 0,
    QCX_ERR_ARG = 1,            /* invalid argument (size, NULL, range)                 */
    QCX_ERR_ALLOC = 2,          /* device or host allocation failed                     */
    QCX_ERR_CUDA = 3,           /* a CUDA runtime/driver call failed                    */
    QCX_ERR_SINGULAR = 4,       /* a dielectric matrix had a zero pivot                 */
    QCX_ERR_NOT_CONVERGED = 5,  /* refinement did not reach its residual bound          */
    QCX_ERR_TIMEOUT = 6,        /* a bounded device-side wait gave up                   */
    QCX_ERR_STATE = 7,          /* call made before the state it needs exists           */
    QCX_ERR_UNSUPPORTED = 8     /* input outside what this build handles (see message)  */
} qcx_status;

typedef enum {
    QCX_FP64 = 0,   /* plain FP64 throughout                                                    */
    QCX_MIXED = 1   /* FP32 pair densities kept as three BF16 terms; chi0 on the tcgen05
                       tensor cores with rho~ = the first two terms on one side and W rho~
                       in three BF16 terms on the other (five products), the FP32
                       tensor-core sums restarted every 20 MMAs and accumulated in FP64, the
                       diagonal summed again from the three-term rho in FP32; eps stored in FP64;
                       FP32 Gauss-Jordan inverse with an FP64 residual correction of the diagonal
                       for ill-conditioned blocks (kappa_1 above qcx_set_refine_threshold, 1e4
                       by default) and the other blocks' loss as a quadratic form of the FP64
                       matrix's anti-Hermitian part; dE and w -+ dE in FP64                    */
} qcx_precision;

typedef struct { double re, im; } qcx_c64;

/* Halo and detector parameters of the nonrelativistic rate (Sec. II.B, IV.B
 * footnote; Appendix A).  m_med_eV < 0 selects the heavy-mediator limit
 * F_DM = 1, m_med_eV == 0 the light limit (alpha m_e / q)^2, otherwise the
 * full form factor of Eq. (F_DM).  The ionisation model is the step
 * Q(w) = 1 + floor((w - w_gap)/w_pp) for w >= w_gap. */
typedef struct {
    double m_chi_eV;          /* dark-matter mass                         */
    double sigma_e_cm2;       /* reference cross section sigma_e          */
    double rho_chi_GeV_cm3;   /* local dark-matter density                */
    double v0_kms;            /* Maxwellian velocity dispersion parameter */
    double vesc_kms;          /* galactic escape speed                    */
    double vE_kms;            /* Earth speed in the galactic frame        */
    double rho_T_g_cm3;       /* target mass density                      */
    double m_med_eV;          /* mediator mass (see above)                */
    double w_gap_eV;          /* ionisation threshold                     */
    double w_pp_eV;           /* energy per extra electron-hole pair      */
} qcx_halo_params;

/* ---------------------------------------------------------------- context */
/* Contexts, streams and error reporting are library plumbing; the paper has
 * no counterpart. */

/* Create a context on CUDA device `device` using `cuda_stream` (a
 * cudaStream_t; NULL = a new non-blocking stream owned by the context).
 * Errors: QCX_ERR_ARG (out == NULL), QCX_ERR_CUDA (device unusable or not
 * sm_103), QCX_ERR_ALLOC. */
qcx_status qcx_create(qcx_ctx** out, int device, void* cuda_stream);

/* Free every device buffer the context owns.  NULL is ignored. */
void qcx_destroy(qcx_ctx* ctx);

/* Message of the last failed call on this context ("" if none).  Valid
 * until the next call on the context. */
const char* qcx_last_error(const qcx_ctx* ctx);

/* Wait for all work queued on the context's stream. */
qcx_status qcx_sync(qcx_ctx* ctx);

/* --------------------------------------------------------------- system */

/* Crystal and Gaussian basis (Sec. III: localized Gaussian orbitals).
 * lattice[9]: rows a_1, a_2, a_3 (bohr).  The lattice must be a sublattice
 * of h Z^3 for some spacing h with all three Cartesian axes equal (simple,
 * face-centred and body-centred cubic in the cubic frame); otherwise
 * QCX_ERR_UNSUPPORTED.  atom_xyz[natom][3] (bohr).  Shells: shell_atom[s]
 * in [0, natom), shell_l[s] in {0, 1}, shell_exp[s] > 0 (bohr^-2); an l = 1
 * shell contributes p_x, p_y, p_z in that order, normalised primitives.
 * Replaces any previous basis and drops all states.
 * Errors: QCX_ERR_ARG, QCX_ERR_UNSUPPORTED, QCX_ERR_ALLOC, QCX_ERR_CUDA. */
qcx_status qcx_set_basis(qcx_ctx* ctx, const double* lattice, int natom, const double* atom_xyz,
                         int nshell, const int* shell_atom, const int* shell_l, const double* shell_exp);

/* Number of basis functions n_b of the current basis (0 if none). */
int qcx_nbasis(const qcx_ctx* ctx);

/* Bloch-sum overlap S_mu,nu(k) = <phi_mu k|phi_nu k> for nk points
 * kpts[nk][3] (bohr^-1), written to out_S[nk][nb][nb] (row mu, column nu).
 * This is the G = 0, q = 0 matrix element of Eq. (RPA), used to
 * orthonormalise coefficients.  Errors: QCX_ERR_STATE (no basis), QCX_ERR_ARG. */
qcx_status qcx_overlap(qcx_ctx* ctx, int nk, const double* kpts, qcx_c64* out_S);

/* Bloch coefficients and band energies (Eq. (RPA) states; T = 0, valence
 * f = 2, conduction f = 0).
 *   kpts[nk][3]            initial-state k grid (bohr^-1)
 *   C_k[nk][nb][nv]        valence coefficients at k, column v = band
 *   E_k[nk][nv]            valence energies (Hartree)
 *   qpts[nq][3]            momentum shifts q (the final-state grid is k + q)
 *   C_kq[nq][nk][nb][nc]   conduction coefficients at k + q
 *   E_kq[nq][nk][nc]       conduction energies (Hartree)
 * Coefficients are used as given (orthonormality is the caller's; see
 * qcx_overlap).  Replaces earlier states.  Errors: QCX_ERR_STATE (no
 * basis), QCX_ERR_ARG, QCX_ERR_ALLOC, QCX_ERR_CUDA. */
qcx_status qcx_set_states(qcx_ctx* ctx, int nk, const double* kpts, int nv, const qcx_c64* C_k,
                          const double* E_k, int nq, const double* qpts, int nc, const qcx_c64* C_kq,
                          const double* E_kq);

/* ------------------------------------------------------------ the path */

/* Pair densities for q number iq and the G set G_int[ng][3]
 * (Eq. (RPA) matrix elements; closed-form Gaussian-product integrals with
 * the lattice sum done as separable one-dimensional sums).  The result is
 * kept in the context (FP64 for QCX_FP64; FP32 values stored as three
 * BF16 terms for QCX_MIXED) and, if out_rho != NULL, also written to
 * out_rho[nt][ng] (complex double).  Starts a new q: the context's chi0,
 * eps and loss tables for other q are untouched; those for iq are reset.
 * Errors: QCX_ERR_STATE (no states), QCX_ERR_ARG (iq, ng < 1, ng > 4096),
 * QCX_ERR_ALLOC, QCX_ERR_CUDA. */
qcx_status qcx_pair_density(qcx_ctx* ctx, int iq, int ng, const int* G_int, qcx_precision prec,
                            qcx_c64* out_rho);

/* Pair densities in the optical limit q -> 0 along the direction qhat[3]
 * (Appendix C, Eq. (ol_overlap) and the head and wing formulas after it), for a
 * q number iq that is exactly zero and whose conduction states are at k itself
 * (orthonormal together with the valence states, as eigenvectors of one H(k)).
 * The G != 0 rows are the pair densities of qcx_pair_density at q = 0; the
 * G = 0 row holds the limit of rho_t(0)/|q|,
 *   rho~_t = -i qhat.p_t / dE_t,  p_t = <c k|grad|v k> (m_e = 1),
 * from the momentum matrix of the Bloch sums (closed-form Gaussian gradient
 * integrals, lattice sum kept as for the pair densities), and v^1/2 of that row
 * is sqrt(4 pi) (the |q| factors cancel).  qcx_chi0 / qcx_chi0_spectral,
 * qcx_invert_eps and qcx_loss_function then give the optical-limit matrix
 * (head, wings, body) and its losses; the G = 0 entry of the loss tables is the
 * optical loss along qhat (|q+G| = 0 there).  The momentum matrix is kept in
 * the context while basis and states are unchanged.  qhat need not be
 * normalised.  out_rho as in qcx_pair_density.
 * Errors: QCX_ERR_STATE (no states), QCX_ERR_ARG (q number iq not zero, G = 0
 * not in the list exactly once, qhat zero or non-finite, a transition with
 * dE = 0, the arguments of qcx_pair_density), QCX_ERR_UNSUPPORTED (3 n_b n_v
 * complex values above 227 KB of shared memory), QCX_ERR_ALLOC, QCX_ERR_CUDA. */
qcx_status qcx_pair_density_optical(qcx_ctx* ctx, int iq, int ng, const int* G_int, const double* qhat,
                                    qcx_precision prec, qcx_c64* out_rho);

/* chi0_GG'(q,w) for nw frequencies w[nw] (Hartree) and broadening eta > 0
 * (Eq. (RPA)), followed in the same kernel by the Dyson step
 * eps = 1 - v^1/2 chi0 v^1/2, kept in the context.  Needs
 * qcx_pair_density(iq) in the same precision.  out_chi0[nw][ng][ng]
 * (row G, column G') is optional.  The loss tables of iq from an earlier
 * qcx_invert_eps are reset (they belong to the previous chi0).
 * Errors: QCX_ERR_STATE, QCX_ERR_ARG (nw < 1, eta <= 0, non-finite w),
 * QCX_ERR_ALLOC, QCX_ERR_CUDA, QCX_ERR_TIMEOUT (a pipeline wait gave up;
 * results are invalid). */
qcx_status qcx_chi0(qcx_ctx* ctx, int iq, int nw, const double* w, double eta, qcx_precision prec,
                    qcx_c64* out_chi0);

/* The spectral route to the same chi0 (Eq. (eRPA_spectral): the spectral
 * part of Eq. (RPA), with the principal part from the Kramers-Kronig
 * relations, Section II.D and its footnote).  On the uniform grid
 * E_b = E0 + b step (b = 0 .. nbin-1, Hartree) each transition's delta is
 * shared between its two neighbouring grid points with hat weights
 * (dE_t = E_b + x step, 0 <= x < 1: weight 1 - x to b, x to b + 1), giving the
 * spectral weights
 *   S_b[G][G'] = 2/(N_k V) sum_t phi_b(dE_t) conj(rho_t(G)) rho_t(G'),
 * formed once per q; then
 *   chi0(w) = sum_b S_b [1/(w - E_b + i eta) - 1/(w + E_b + i eta)]
 * (the same retarded broadening as qcx_chi0, so both routes agree exactly
 * when every dE_t lies on the grid and otherwise differ by the interpolation
 * in energy, second order in step) and eps = 1 - v^1/2 chi0 v^1/2 kept in the
 * context like qcx_chi0, for qcx_invert_eps.  Needs qcx_pair_density(iq) in
 * the same precision.  QCX_FP64: FP64 throughout.  QCX_MIXED: FP32 pair
 * densities (the mixed path's), FP32 spectral weights, and the contraction
 * over the grid points on the tcgen05 tensor cores with K and the weights as
 * three-term split BF16 (FP32 sums restarted every 24 MMAs, added in FP32 per
 * chunk of at most 4096 points, chunks added in FP64); grid and K in FP64.
 *   out_chi0[nw][ng][ng]  optional, row G, column G' (complex double)
 *   out_S[nbin][ng][ng]   optional spectral weights (complex double); large
 * Memory: the weights are formed in chunks of grid points (about 4 GiB, or
 * qcx_set_spectral_chunk), plus [ng][nt] grouped pair densities.
 * Errors: QCX_ERR_STATE, QCX_ERR_ARG (nw < 1, eta <= 0, step <= 0, nbin < 2,
 * non-finite w or E0, a dE_t outside [E0, E0 + (nbin - 1) step)),
 * QCX_ERR_UNSUPPORTED (more than 2^31 - 1 transitions), QCX_ERR_ALLOC,
 * QCX_ERR_CUDA. */
qcx_status qcx_chi0_spectral(qcx_ctx* ctx, int iq, int nw, const double* w, double eta, double E0,
                             double step, int nbin, qcx_precision prec, qcx_c64* out_chi0,
                             qcx_c64* out_S);

/* The grid that qcx_chi0_spectral needs for q number iq at spacing step:
 * E0 = step floor(min dE / step) - step, nbin = floor((max dE - E0)/step) + 3,
 * so every transition lies inside with one spare point on each side.
 * Errors: QCX_ERR_STATE (no states), QCX_ERR_ARG (step <= 0, non-finite
 * energies, more than 2^30 points), QCX_ERR_CUDA. */
qcx_status qcx_spectral_grid(qcx_ctx* ctx, int iq, double step, double* E0, int* nbin);

/* Grid points per chunk of qcx_chi0_spectral (rounded down to a multiple of
 * 32, at least 32); 0 (default) takes them from a 4 GiB budget for the
 * chunk's spectral weights.  Results do not depend on it beyond rounding
 * (chunks are added in FP64).  Errors: QCX_ERR_ARG (ctx NULL, bins < 0). */
qcx_status qcx_set_spectral_chunk(qcx_ctx* ctx, int bins);

/* Engine of the mixed route's contraction in qcx_chi0_spectral: 0 (default)
 * the tcgen05 tensor cores, nonzero the CUDA cores in FP32 (partial sums over
 * 64 grid points added into a second FP32 sum), kept for comparison.  Library
 * plumbing.  Errors: QCX_ERR_ARG (ctx NULL). */
qcx_status qcx_set_spectral_engine(qcx_ctx* ctx, int cuda_cores);

/* Device times (ms, CUDA events on the context's stream) of the stages of the
 * last qcx_chi0_spectral call: ms[0] grouping of the transitions by grid
 * point, ms[1] gather of the pair densities and the K table, ms[2] spectral
 * weights, ms[3] Kramers-Kronig contraction, ms[4] Dyson step (zeros before
 * the first call).  Library plumbing, no counterpart in the paper.
 * Errors: QCX_ERR_ARG (ctx or ms NULL). */
qcx_status qcx_spectral_timings(qcx_ctx* ctx, double* ms);

/* Inverse of every eps(w) of the last qcx_chi0(iq) call: Gauss-Jordan with
 * partial pivoting (FP64; for QCX_MIXED FP32 followed, where the block is
 * ill-conditioned, by one FP64 residual correction of the diagonal).
 * Writes, if not NULL,
 *   out_diag_inv[nw][ng]   [eps^-1]_GG                     (Eq. (eps_LFE))
 *   out_eps_diag[nw][ng]   eps_GG                          (Eq. (eps_noLFE))
 *   out_resid[nw]          QCX_MIXED: max_G |correction| / |[eps^-1]_GG| of the
 *                          FP64 correction for blocks with kappa_1 above the
 *                          threshold of qcx_set_refine_threshold (the
 *                          ill-conditioned ones), 0 for the others; 0 for QCX_FP64.
 * and keeps the loss tables of iq in the context.
 * Errors: QCX_ERR_STATE, QCX_ERR_SINGULAR (zero pivot in some block; the
 * other blocks are valid), QCX_ERR_ALLOC, QCX_ERR_CUDA. */
qcx_status qcx_invert_eps(qcx_ctx* ctx, int iq, qcx_precision prec, qcx_c64* out_diag_inv,
                          qcx_c64* out_eps_diag, double* out_resid);

/* A setting of the mixed path of qcx_invert_eps (no counterpart in the
 * paper; the loss it serves is Eq. (eps_LFE)): blocks whose condition estimate
 * kappa_1 = |eps|_1 |X|_1 (X the FP32 inverse) exceeds kappa1 get the FP64
 * correction of the diagonal (the precision plan's FP64 residual near the
 * plasmon, where eps is ill-conditioned); the others take L_LFE as the
 * diagonal of X B X^H with B = (eps - eps^H)/(2i), formed from the FP64 eps.
 * Default 1e4; 0 corrects every block.  Applies to later qcx_invert_eps calls
 * of this context.  Errors: QCX_ERR_ARG (ctx NULL, kappa1 negative or NaN). */
qcx_status qcx_set_refine_threshold(qcx_ctx* ctx, double kappa1);

/* Failure handling, no counterpart in the paper: every wait inside the
 * tensor-core chi0 kernels (qcx_chi0 with QCX_MIXED, and the batch plans of
 * qcx_solve_batch built after this call) gives up after `cycles` SM clock
 * cycles (default 4e9, about 2 s); the kernel then stops its pipeline, lets its
 * own copies and MMAs finish, frees its tensor memory and returns, and the
 * call reports QCX_ERR_TIMEOUT with invalid results while the context stays
 * usable.  A short limit makes the waits run out on purpose (tests).
 * Errors: QCX_ERR_ARG (ctx NULL, cycles < 1). */
qcx_status qcx_set_wait_limit(qcx_ctx* ctx, long long cycles);

/* Fault injection for tests of the failure path (no counterpart in the
 * paper): with withhold_copies != 0 the tensor-core kernel of qcx_chi0
 * (QCX_MIXED) issues none of its copies, so its consumers' waits run out after
 * the limit of qcx_set_wait_limit and the call returns QCX_ERR_TIMEOUT; 0
 * (the default) restores normal operation.  Errors: QCX_ERR_ARG (ctx NULL). */
qcx_status qcx_set_fault_injection(qcx_ctx* ctx, int withhold_copies);

/* Loss functions of q number iq (Eq. (dynamic_structure_factor)):
 *   out_L_lfe[nw][ng]   = -Im [eps^-1]_GG   (with local fields)
 *   out_L_nolfe[nw][ng] = -Im (1/eps_GG)    (without)
 * Needs qcx_invert_eps(iq) after the last qcx_pair_density(iq) and
 * qcx_chi0(iq) (and after the last qcx_set_states); the tables stay until
 * then.  Errors: QCX_ERR_STATE (tables not current), QCX_ERR_CUDA. */
qcx_status qcx_loss_function(qcx_ctx* ctx, int iq, double* out_L_lfe, double* out_L_nolfe);

/* Average the stored loss tables of the listed q over |q+G| bins
 * (momentum q + G carries [eps^-1]_GG by Eq. (eps_LFE)).  which = 0: with
 * local fields, 1: without.  edges[nbin+1] ascending (bohr^-1).  All listed
 * q must share nw and the frequency grid.  out_L[nbin][nw] is the bin mean
 * (0 for empty bins), out_count[nbin] the number of (q, G) per bin.
 * Errors: QCX_ERR_STATE (a q without loss table), QCX_ERR_ARG. */
qcx_status qcx_bin_loss(qcx_ctx* ctx, int nsel, const int* iq_list, int which, int nbin,
                        const double* edges, double* out_L, double* out_count);

/* Nonrelativistic halo rate dR/dw = (rho_chi/m_chi)(1/rho_T) sigma_e/(8 pi^2
 * alpha mu^2) int dq q^3 |F_DM|^2 L(w,q) eta(v_min) (end of Appendix A with
 * Eqs. (general_rate), (v_min)), composite trapezoid over qbin[nqbin]
 * (ascending, bohr^-1) with L[nqbin][nw]; w[nw] uniform (Hartree).
 * out_dRdw[nw] in events/(kg yr eV); out_dRQ[nQ] = sum_w dR/dw dw over
 * Q(w) = 1..nQ (Eq. (excitation_rate)) in events/(kg yr).  Accumulation in
 * FP64.  Errors: QCX_ERR_ARG. */
qcx_status qcx_rate(qcx_ctx* ctx, int nqbin, const double* qbin, int nw, const double* w,
                    const double* L, const qcx_halo_params* params, double* out_dRdw, int nQ,
                    double* out_dRQ);

/* ------------------------------------------------ rate end: 3-D tables */

/* The composite dielectric function binned in three-dimensional momentum
 * space (Section III, Eq. (e_comp)): for the listed q (their qcx_invert_eps
 * tables, same frequency grid) every value eps(w, q+G) is taken as
 * eps^LFE = 1/[eps^-1]_GG (Eq. (eps_LFE), with the imaginary part of
 * [eps^-1]_GG the stored -L_LFE) where |q+G| <= q_lfe and as
 * eps^noLFE = eps_GG (Eq. (eps_noLFE)) above it, and falls in shell
 * floor(|q+G|/dq) (< nshell), polar cell floor(theta n_theta/pi) and azimuthal
 * cell floor(phi n_phi/(2 pi)) with phi in [0, 2 pi) (edge values to the last
 * cell).  Writes the bin means out_eps[nshell][n_theta][n_phi][nw] and the
 * numbers of values out_count[nshell][n_theta][n_phi] (empty: 0).  With
 * fill != 0 an empty bin lying between filled shells of the same angular cell
 * takes the linear interpolation in |q| of the nearest filled shells on either
 * side and its count is set to -1.  Lengths in bohr^-1; outputs host or device.
 * Errors: QCX_ERR_STATE (a q without loss tables), QCX_ERR_ARG (sizes, grids
 * that differ, dq <= 0), QCX_ERR_ALLOC, QCX_ERR_CUDA. */
qcx_status qcx_bin_eps3d(qcx_ctx* ctx, int nsel, const int* iq_list, double q_lfe, int nshell, double dq,
                         int n_theta, int n_phi, int fill, qcx_c64* out_eps, double* out_count);

/* Screening of the loss function (Section IV.C): Im(-1/eps)_scr =
 * Im eps / |eps_scr|^2 (Eq. (ELF_screening)) with eps_scr = eps itself
 * (QCX_SCREEN_SELF: the loss function Im(-1/eps)), 1 (QCX_SCREEN_NONE), the
 * modified Thomas-Fermi model (QCX_SCREEN_MTF, Eq. (MTF); eps0, tau, wp_eV,
 * qtf_eV) or the Lindhard function of an electron gas of density ne_bohr3 with
 * damping f_p (QCX_SCREEN_LINDHARD, Eq. (Lindhard); fp > 0). */
#define QCX_SCREEN_SELF 0
#define QCX_SCREEN_NONE 1
#define QCX_SCREEN_MTF 2
#define QCX_SCREEN_LINDHARD 3
typedef struct {
    int model;
    double eps0, tau, wp_eV, qtf_eV;   /* modified Thomas-Fermi parameters */
    double ne_bohr3, fp;               /* Lindhard: electron density (bohr^-3), damping fraction of w_p */
} qcx_screening;

/* Isotropic loss function of 3-D tables (as from qcx_bin_eps3d):
 * out_L[nshell][nw] = mean over the angular cells of each shell with
 * count != 0 of Im eps_cell / |eps_scr|^2, the screening models evaluated at
 * the shell centre |q| = (s + 1/2) dq and at w[nw] (Hartree);
 * out_ncell[nshell] = cells used (0: L = 0).  Inputs and outputs host or
 * device.  Errors: QCX_ERR_ARG (sizes, unknown model, fp <= 0 for Lindhard),
 * QCX_ERR_ALLOC, QCX_ERR_CUDA. */
qcx_status qcx_loss_isotropic(qcx_ctx* ctx, int nshell, int n_theta, int n_phi, int nw, const double* w,
                              double dq, const qcx_c64* eps, const double* count, const qcx_screening* scr,
                              double* out_L, double* out_ncell);

/* Particle and mediator of the general rate. */
typedef struct {
    double m_chi_eV;          /* dark-matter mass                                         */
    double sigma_e_cm2;       /* reference cross section sigma_e                          */
    double m_med_eV;          /* mediator mass: < 0 heavy limit, 0 massless, > 0 the mass */
    int mediator;             /* 0 vector, 1 scalar (Eq. (H))                            */
    double rho_T_g_cm3;       /* target mass density                                      */
    double w_gap_eV, w_pp_eV; /* ionisation step model Q(w) = 1 + floor((w - w_gap)/w_pp) */
    double exposure_kg_yr;    /* reach: exposure ...                                      */
    double n_events;          /* ... and expected events (2.3: zero background, 90 % CL) */
} qcx_rate_params;

/* General rate for a velocity flux (Eqs. (general_rate), (H),
 * (cross_section_iso), (v_min)): dR/dw = (1/rho_T) int dv dPhi/dv
 * sigma_e/(16 pi mu^2) 1/(E (E - w)) int dq q H(q) F(w, q) S(w, q)
 * Theta(v - v_min)/v^2 with S = q^2 L/(2 pi alpha), E = gamma m_chi,
 * v_min = q/(2 gamma m_chi) + w/q and F = (m^2 + (alpha m_e)^2)^2/(w^2 - q^2 - m^2)^2
 * (1 in the heavy limit); transfers with E - w <= m_chi contribute 0.
 * qbin[nqbin] (bohr^-1, ascending) and L[nqbin][nw], w[nw] (Hartree, uniform),
 * v[nv] (units of c, ascending) with dphidv[nv] (1/(cm^2 s) per unit v); both
 * integrals by the composite trapezoid, accumulation in FP64.  Writes
 * out_dRdw[nw] (events/(kg yr eV)), out_dRQ[nQ] (events/(kg yr) per
 * ionisation step, Eq. (excitation_rate)) and, if not NULL, out_reach[nQ]:
 * the cross section at which n_events are expected above threshold Q in the
 * exposure.  Errors: QCX_ERR_ARG. */
qcx_status qcx_rate_general(qcx_ctx* ctx, int nqbin, const double* qbin, int nw, const double* w, const double* L,
                            int nv, const double* v, const double* dphidv, const qcx_rate_params* params,
                            double* out_dRdw, int nQ, double* out_dRQ, double* out_reach);

/* --------------------------------------------------- batched instances */

/* Uneven (q, w) instances in one call: instance i is the frequency
 * inst_w[i] (Hartree) of the q point inst_q[i] (an index into the q list of
 * qcx_set_states) with its own G set {G : |q + G| < inst_gmax[i]} (bohr^-1),
 * and yields the heads of the loss functions (Eq. (RPA) with the Dyson step;
 * Eq. (eps_LFE) and Eq. (eps_noLFE) at G = 0):
 *   out_L_lfe_head[i]   = -Im [eps^-1]_{00}
 *   out_L_nolfe_head[i] = -Im (1 / eps_00)
 *   out_ng[i]           = N_G of the instance (may be NULL).
 * eta (Hartree) is shared.  QCX_FP64 computes everything in FP64; QCX_MIXED
 * forms chi0 on the tensor cores (split-BF16 products as for qcx_chi0, FP32
 * accumulation promoted to FP64, eps in FP64), factors eps in FP32 (LU, partial pivoting)
 * and refines the head with two FP64-residual correction steps.
 * The first call with a new instance list (same q indices, cutoffs, eta and
 * precision) plans the batch: G sets, pair densities once per distinct q on
 * the union of its instances' sets, tile and per-SM instance lists; for
 * QCX_MIXED it also times one CUDA graph per tile width and keeps the fastest
 * (see qcx_batch_autotune).  The whole batch then runs as one captured CUDA
 * graph (a single persistent tensor-core launch per 16 distinct q), replayed
 * by later calls with the same list; only the frequencies may change between
 * them.  The plan holds its own device buffers until the next plan, new
 * states or qcx_destroy.  Inputs: host or device pointers; outputs: host or
 * device pointers (the call synchronises the context stream).
 * Errors: QCX_ERR_STATE (no states), QCX_ERR_ARG (sizes, q index, non-finite
 * or non-positive cutoff, or G = 0 outside an instance's cutoff),
 * QCX_ERR_UNSUPPORTED (an instance with N_G > 512), QCX_ERR_SINGULAR (zero
 * pivot: that instance's L_LFE is 0), QCX_ERR_NOT_CONVERGED (QCX_MIXED: the
 * last correction exceeded 1e-6 relative), QCX_ERR_TIMEOUT (a bounded wait in
 * the tensor-core kernel gave up; results invalid), QCX_ERR_ALLOC,
 * QCX_ERR_CUDA.  Outputs are written in every case except ARG, STATE,
 * UNSUPPORTED, ALLOC and CUDA errors. */
qcx_status qcx_solve_batch(qcx_ctx* ctx, int ninst, const int* inst_q, const double* inst_w,
                           const double* inst_gmax, double eta, qcx_precision prec, double* out_L_lfe_head,
                           double* out_L_nolfe_head, int* out_ng);

/* Facts about the current batch plan (batching has no counterpart in the
 * paper), written to out[0 .. n-1] (host):
 * [0] tile width cap (columns of G per tensor-core tile), [1] tiles,
 * [2] persistent tensor-core CTAs, [3] solve CTAs, [4] kernels per replay,
 * [5] 1 if the tile widths were autotuned, [6] distinct q, [7] largest N_G,
 * [8] autotuning time (microseconds), [9] precision, [10..12] the tile width
 * caps of the N_G classes 65-128, 129-192 and above 192 ([0] repeats the last).
 * Entries past 12 are 0.
 * Errors: QCX_ERR_ARG, QCX_ERR_STATE (no plan yet; out is zeroed). */
qcx_status qcx_batch_info(const qcx_ctx* ctx, int n, long long* out);

/* Turn the tile-width autotuning of new QCX_MIXED batch plans on (default)
 * or off (then the widest tiles, caps of 192, are used); no counterpart in the paper.  Errors: QCX_ERR_ARG (ctx NULL). */
qcx_status qcx_batch_autotune(qcx_ctx* ctx, int enable);

/* ----------------------------------------- learned local-field correction */

/* A surrogate that the paper does not have: a network
 * 6 -> 128 -> 128 -> 128 -> 2 (SiLU hidden activations) that maps the inputs
 *   x = (|q| / q_max, q / |q| (3 components), w / w_max, ln(L_noLFE) / 10)
 * of one (q, w) head to (mu, s): mu estimates y = log(L_LFE / L_noLFE) and
 * s = log sigma^2 its uncertainty, so that L_LFE ~ L_noLFE e^mu can stand in
 * for the Dyson route where sigma is small, with the Dyson route (the heads
 * of qcx_solve_batch or of qcx_invert_eps) as fallback and check.
 * Parameters: one FP32 vector of QCX_MLP_NPARAM = 34178 entries, per layer
 * W [out][in] row-major then b [out] (layers 6->128, 128->128, 128->128,
 * 128->2).  Compute copies of the weight matrices are BF16; biases,
 * activations, accumulations and gradients FP32.  Training minimises the
 * Gaussian negative log-likelihood (s + (y - mu)^2 e^-s) / 2 averaged over
 * each step's samples with Adam (bias-corrected), FP32 moments. */
#define QCX_MLP_NPARAM 34178

typedef struct {
    int epochs;              /* passes over the data                              */
    int batch;               /* samples per Adam step (last step of a pass: rest) */
    float lr, beta1, beta2, eps;
    unsigned long long seed; /* shuffle of each pass (Fisher-Yates, SplitMix64)   */
} qcx_mlp_opts;

/* QCX_MLP_NPARAM (for bindings). */
int qcx_mlp_nparam(void);

/* Load the FP32 parameters (host or device, QCX_MLP_NPARAM floats), refresh
 * the BF16 copies and reset the Adam moments and step count.
 * Errors: QCX_ERR_ARG (NULL, non-finite entry), QCX_ERR_ALLOC, QCX_ERR_CUDA. */
qcx_status qcx_mlp_set_params(qcx_ctx* ctx, const float* params);

/* Copy out the FP32 parameters and (if out_compute != NULL) the values the
 * kernels compute with (BF16 weights widened to FP32, FP32 biases); either
 * pointer may be host or device, QCX_MLP_NPARAM floats each.
 * Errors: QCX_ERR_STATE (no parameters), QCX_ERR_CUDA. */
qcx_status qcx_mlp_get_params(qcx_ctx* ctx, float* out_params, float* out_compute);

/* Gradient of the mean loss over n samples X[n][6], y[n] with respect to
 * the parameters (written to out_grad[QCX_MLP_NPARAM]) and the mean loss
 * (out_loss, host, may be NULL).  No update.  Errors: QCX_ERR_STATE,
 * QCX_ERR_ARG, QCX_ERR_ALLOC, QCX_ERR_CUDA. */
qcx_status qcx_mlp_grad(qcx_ctx* ctx, int n, const float* X, const float* y, float* out_grad, double* out_loss);

/* Train on X[n][6], y[n] (host or device) for opts->epochs shuffled passes;
 * the pass is captured once as a CUDA graph and replayed.  out_epoch_loss
 * (host, may be NULL) receives the mean loss of each pass (computed during
 * the pass).  Errors: QCX_ERR_STATE, QCX_ERR_ARG, QCX_ERR_ALLOC,
 * QCX_ERR_CUDA, QCX_ERR_NOT_CONVERGED (the loss became non-finite). */
qcx_status qcx_mlp_train(qcx_ctx* ctx, int n, const float* X, const float* y, const qcx_mlp_opts* opts,
                         float* out_epoch_loss);

/* (mu, s) for X[n][6]; outputs host or device.  Errors: QCX_ERR_STATE,
 * QCX_ERR_ARG, QCX_ERR_ALLOC, QCX_ERR_CUDA. */
qcx_status qcx_mlp_predict(qcx_ctx* ctx, int n, const float* X, float* out_mu, float* out_logvar);

/* The surrogate route for the heads.  qcx_head_nolfe: L_noLFE at the head
 * of q number iq for nw frequencies (Hartree, host or device), from
 * Eq. (eps_noLFE) at G = 0: eps_00 = 1 - v(q) chi0_00 with chi0_00 = 2/(N_k V) sum_t W_t |rho_t(q)|^2
 * in FP64 (only rho at G = 0 is formed).  It uses the context's FP64 per-q
 * state, so a later qcx_chi0 needs qcx_pair_density again.
 * Errors: QCX_ERR_STATE, QCX_ERR_ARG (q = 0 among them), QCX_ERR_ALLOC,
 * QCX_ERR_CUDA. */
qcx_status qcx_head_nolfe(qcx_ctx* ctx, int iq, int nw, const double* w, double eta, double* out_L_nolfe_head);

/* Network inputs X[n][6] (FP32) from q vectors qvec[n][3] (bohr^-1),
 * frequencies w[n] (Hartree) and L_noLFE[n]: (|q|/q_max, q/|q|, w/w_max,
 * ln(L_noLFE)/10); with L_lfe[n] also the training targets
 * out_y[n] = log(L_LFE / L_noLFE) (L_lfe and out_y both NULL or both set).
 * Inputs and outputs host or device.  Errors: QCX_ERR_ARG, QCX_ERR_ALLOC,
 * QCX_ERR_CUDA. */
qcx_status qcx_surrogate_features(qcx_ctx* ctx, int n, const double* qvec, const double* w, const double* L_nolfe,
                                  const double* L_lfe, double q_max, double w_max, float* out_X, float* out_y);

typedef struct {
    double q_max, w_max;       /* feature scaling (bohr^-1, Hartree), as in training          */
    double sigma_accept;       /* accept where e^(s/2) < sigma_accept                        */
    double check_frac;         /* fraction of accepted samples re-solved by the Dyson route  */
    double check_tol;          /* spot check passes if |mu - log(L_LFE/L_noLFE)| <= check_tol */
    unsigned long long seed;   /* choice of the spot-checked samples                          */
} qcx_surrogate_opts;

/* Heads for nsel q points (indices iq_list) x nw frequencies w (host), the
 * Dyson route on the G list G_int[ng][3] (host; must contain G = 0) being the
 * fallback: per sample the network predicts (mu, s) from qcx_head_nolfe's
 * L_noLFE; L_LFE = L_noLFE e^mu is kept where e^(s/2) < sigma_accept; a
 * seeded fraction check_frac of the kept samples is re-solved by the Dyson
 * route (fallback_prec) and if any misses by more than check_tol in
 * |log ratio| all samples fall back; rejected samples always take the Dyson
 * route.  Outputs [nsel][nw] (host or device; L_nolfe and source may be
 * NULL): out_L_lfe_head, out_L_nolfe_head, out_source (0 surrogate,
 * 1 Dyson route, 2 Dyson route as a spot check), out_check_err (host: the
 * largest spot-check miss, -1 if none was checked).  Replaces the context's
 * per-q state.  Errors: QCX_ERR_STATE (no states or no network parameters),
 * QCX_ERR_ARG, QCX_ERR_SINGULAR, QCX_ERR_ALLOC, QCX_ERR_CUDA. */
qcx_status qcx_surrogate_heads(qcx_ctx* ctx, int nsel, const int* iq_list, int ng, const int* G_int, int nw,
                               const double* w, double eta, qcx_precision fallback_prec,
                               const qcx_surrogate_opts* opts, double* out_L_lfe_head, double* out_L_nolfe_head,
                               int* out_source, double* out_check_err);

/* ------------------------------------------------------- no allocation */

/* The paper has no counterpart to this entry point; it exists for callers
 * that cannot allocate device memory when they need the result: a framework
 * that owns the device allocator and forbids other libraries from calling
 * cudaMalloc (which also synchronises the device, something a latency-bound
 * or graph-replayed pipeline cannot afford), or a process that reserved its
 * whole memory budget at start-up.  It computes what qcx_invert_eps computes
 * for QCX_FP64 (Gauss-Jordan with partial pivoting in FP64) for nb
 * caller-owned dielectric matrices, and allocates nothing:
 *   eps[nb][n][n]           device, complex FP64, row-major (row G, column G')
 *   out_diag_inv[nb][n]     device: [eps^-1]_GG
 *   out_L_lfe[nb][n]        device or NULL: -Im [eps^-1]_GG
 *   out_L_nolfe[nb][n]      device or NULL: -Im (1/eps_GG)
 *   out_singular[nb]        device or NULL: 1 where a zero pivot was met
 *                           (that matrix's outputs are then zero), else 0
 *   cuda_stream             stream to run on (NULL = legacy default stream)
 * The only scratch is a fixed 16 MiB device array inside the library: calls
 * need nb * n * n * 16 bytes <= 16 MiB, otherwise QCX_ERR_ARG and nothing
 * runs.  A device reserves the array when it loads the code of this entry
 * point; under CUDA's default lazy module loading (CUDA_MODULE_LOADING=LAZY)
 * that is this entry point's first call on the device, which also resolves
 * the array's address for that device (cudaGetSymbolAddress with the device
 * current).  The array is then held until the process exits.  So make the
 * first call on each device before reserving the rest of the memory budget,
 * and outside any stream capture; that call can fail with QCX_ERR_CUDA when
 * the device has no 16 MiB left.  Every call shares the array and leaves its last
 * contents there; every element a call uses is written by that call first,
 * so nothing needs clearing.  Calls that overlap on the GPU (on different
 * streams, or from different threads) race on the array: serialise them.
 * No cudaMalloc, cudaFree or allocating library routine is called.  The call
 * is asynchronous on cuda_stream.
 * Errors: QCX_ERR_ARG (sizes, a non-device pointer, over the scratch limit),
 * QCX_ERR_CUDA (no usable device, launch failure). */
qcx_status qcx_eps_inverse_diag_noalloc(const qcx_c64* eps, int nb, int n, qcx_c64* out_diag_inv,
                                        double* out_L_lfe, double* out_L_nolfe, int* out_singular,
                                        void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* QCX_H */
