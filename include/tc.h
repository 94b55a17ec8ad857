/*
 * tc.h -- C ABI of the GB300 transcorrelated (TC / BITC) interaction operator.
 *
 * The library applies the effective two-body and three-body interactions of
 * the TC Hamiltonian (M. Ochi, arXiv:2302.07420, Sec. 2.1, Eqs. V2body and
 * V3body; the three-body part contracted over occupied orbitals as in
 * Eq. SCF / Eq. BITCSCF) to every right orbital phi and every left orbital chi
 * at every k-point, including the divergence corrections for k-points on the
 * SCF mesh (Sec. 2.5 and the corrections listed in Sec. 2.6.4).  One spin
 * channel is computed (non-spin-polarised: both channels hold the same
 * orbitals); same-spin pairs use the parallel-spin Jastrow (A[0], C[0]) and
 * opposite-spin pairs the antiparallel one (A[1], C[1]).
 *
 * Units: Hartree atomic units.  Orbitals are given by their plane-wave
 * coefficients c(G) on the sphere |k+G|^2/2 <= ecut_ha, normalised so that
 * sum_G |c(G)|^2 = 1 (phi_periodic(r) = sum_G c(G) e^{iG.r} / sqrt(Omega),
 * Sec. 2.3).  Outputs are coefficients in the same units on the same sphere.
 *
 * Layout of every orbital array: interleaved complex FP64
 * [Nk][nbands][npw_max] (real, imaginary), zero padded beyond npw(k), in the
 * k and G order reported by tc_layout: k index (i1*N2 + i2)*N3 + i3 of the
 * Gamma-centred mesh with fractional coordinates in (-1/2, 1/2]; G order
 * lexicographic in the Miller indices (m1, m2, m3).
 *
 * Pointers: orbital arrays may be device pointers or host pointers (pageable
 * or pinned); host arrays are staged through the library's own device buffers
 * on the given stream, so a call with host pointers includes the copies and
 * returns after the outputs have landed.  occ is always a host array.
 *
 * Ownership: the caller owns every buffer it passes.  The context owns its
 * tables and workspace, all allocated in tc_init; tc_apply / tc_energy
 * allocate nothing (tc_apply_noalloc needs no context at all).
 *
 * Errors: no call aborts or throws across the ABI.  On a non-OK status the
 * contents of the output arrays are undefined; tc_last_error gives the reason.
 * Fault injection (host only, for testing a caller's error handling; the
 * paper has no counterpart): the environment variable TC_FAULT, read on every
 * call, makes tc_init and tc_init_batch return TC_ERR_OOM before any device
 * allocation (TC_FAULT=alloc), and tc_apply, tc_energy, tc_energy_grad,
 * tc_autotune, tc_davidson_step, tc_apply_batch and tc_apply_noalloc return
 * TC_ERR_CUDA (TC_FAULT=launch) or TC_ERR_TIMEOUT (TC_FAULT=timeout) before
 * any kernel launch, with the outputs untouched and the context usable.
 * TC_FAULT=nocluster makes tc_init treat every thread-block-cluster pair
 * kernel as one the device cannot hold (as cudaOccupancyMaxActiveClusters
 * reporting 0 would): its contexts run the one-CTA kernels with full
 * transforms instead (tc_pair_kernels reports it; results equal to rounding).
 * TC_ERR_TIMEOUT is otherwise not returned: no kernel of this library waits
 * on a flag or on another kernel.
 * Threads: a context is not thread-safe; distinct contexts are independent.
 * Streams: work is enqueued on the CUDA stream passed (cudaStream_t, NULL =
 * legacy default stream).  Calls with device pointers return without
 * synchronising (except tc_energy, which returns host scalars).
 */
#ifndef TC_GB300_H
#define TC_GB300_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  TC_OK = 0,
  TC_ERR_ARG = 1,          /* invalid argument (null pointer, bad size, bad parameter) */
  TC_ERR_STATE = 2,        /* context not initialised or already destroyed */
  TC_ERR_OOM = 3,          /* device or host allocation failed (tc_init only) */
  TC_ERR_CUDA = 4,         /* a CUDA runtime call or kernel launch failed */
  TC_ERR_TIMEOUT = 5,      /* a bounded device wait gave up (only injected: see TC_FAULT) */
  TC_ERR_UNSUPPORTED = 6,  /* valid but not supported (e.g. FFT box size) */
  TC_ERR_NUMERIC = 7       /* a numerical step failed (vanishing norm, singular overlap,
                              eigen-solver without convergence); outputs undefined */
} tc_status;

/* Precision of the FFTs and pair products (the energy sums, overlaps and divergence-correction
 * scalars are FP64 in every mode; Sec. 2.6 prints no precision, the FP64 path is the reference).
 *   TC_FP64        FP64 fields and transforms.
 *   TC_FP32        FP32 fields and transforms, FP32 accumulation (in L2 reductions, fixed order).
 *   TC_FP32_COMP   FP32 with compensated accumulation: not built, tc_init returns
 *                  TC_ERR_UNSUPPORTED (plain FP32 accumulation already meets the 1e-5 bound of
 *                  the operator output with a wide margin).
 *   TC_BF16_STORE  TC_FP32 with the real-space orbital fields (phi, chi and their gradients,
 *                  the operands of every pair density) rounded to BF16 (8-bit mantissa,
 *                  round to nearest even) when they are stored; they are held in FP32 words and
 *                  every product, transform and sum runs in FP32.  Its error (about 2^-9 per
 *                  field value) is reported against FP64; it does not meet the 1e-5 bound. */
enum { TC_FP64 = 0, TC_FP32 = 1, TC_FP32_COMP = 2, TC_BF16_STORE = 3 };

/* Term indices of the operator (Sec. 2.6.3-2.6.4) and of E_terms.  The
 * three-body outputs include their multiplicities: 3a3 and 3a4 twice (3a6 = 3a3,
 * 3a5 = 3a4), every 3b term twice (3c = 3b). */
enum {
  TC_TERM_2AH = 0, TC_TERM_2BH1, TC_TERM_2BH2, TC_TERM_2AX, TC_TERM_2BX1, TC_TERM_2BX2,
  TC_TERM_3A1, TC_TERM_3A2, TC_TERM_3A3, TC_TERM_3A4,
  TC_TERM_3B1, TC_TERM_3B2, TC_TERM_3B3, TC_TERM_3B4, TC_TERM_3B5, TC_TERM_3B6,
  TC_NTERMS_OP,                 /* 16 operator terms */
  TC_TERM_KIN = TC_NTERMS_OP,   /* kinetic energy (energy breakdown only) */
  TC_NTERMS                     /* 17 entries in E_terms */
};

typedef struct {
  double lattice[3][3];   /* bohr, rows a_1, a_2, a_3 */
  int kmesh[3];           /* Gamma-centred Monkhorst-Pack mesh */
  double ecut_ha;         /* plane-wave sphere |k+G|^2/2 <= ecut_ha (Hartree) */
  int fft[3];             /* FFT box; cubic, n in {9, 12, 15, 16, 18, 20, 24, 25, 27, 30, 32, 48} */
  int nbands;             /* bands per k (outputs) */
  int nocc;               /* occupied bands per k (partners), 0 < nocc <= nbands */
  double A[2];            /* Jastrow A (Eq. Jastrow) for [parallel, antiparallel] spins */
  double C[2];            /* Jastrow C for [parallel, antiparallel] spins, > 0 */
  double alpha;           /* auxiliary-function exponent (Eq. aux); <= 0 selects
                             sqrt(alpha) = (shortest supercell vector) / 12 */
  int div_correction;     /* 1: add the SCF-mesh divergence corrections (default) */
  double ushort_factor;   /* factor on the u_short terms of Eqs. divcor_3a2_first and
                             3b6_div_scf1; 1 reproduces the printed equations */
  int precision;          /* TC_FP64, TC_FP32 or TC_BF16_STORE (TC_FP32_COMP: unsupported) */
  unsigned int term_mask; /* bit t enables operator term t; 0 enables all */
} tc_params;

typedef struct tc_ctx tc_ctx;

/* Builds cell, Gamma-centred k mesh and plane-wave spheres (Sec. 2.3), box
 * maps, the FP64 kernel tables of V_2a, V_2a^dagger and u~ at every distinct
 * k - q + G (Sec. 2.6.3, Appendix B) and the divergence-correction constant
 * Gamma0 (Eq. correction2, Sec. 2.5) on the host, then uploads them and
 * allocates all device workspace on the current CUDA device (tc_apply and
 * tc_energy allocate nothing).  *out is owned by the caller and released by
 * tc_destroy.  Errors (reason in tc_last_error(NULL), *out = NULL):
 * TC_ERR_ARG (invalid parameters, a sphere that does not fit the box),
 * TC_ERR_UNSUPPORTED (box size without a compiled specialisation, non-cubic
 * box), TC_ERR_OOM (device allocation), TC_ERR_CUDA. */
tc_status tc_init(const tc_params* params, tc_ctx** out);

/* Basis layout.  *npw_per_k -> [Nk] ints, *miller -> [Nk][npw_max][3] ints
 * (zero padded); both pointers stay valid until tc_destroy.  Any output
 * pointer may be NULL. */
tc_status tc_layout(const tc_ctx* ctx, int* nk, int* npw_max, const int** npw_per_k, const int** miller);

/* Scalars of the setup: out[0] = Omega, out[1] = alpha, out[2] = Gamma0 (the
 * bracket of Eq. correction2), out[3] = number of distinct k - q vectors. */
tc_status tc_setup_scalars(const tc_ctx* ctx, double out[4]);

/* out_R = (h_2 + h_3) phi_j and out_L = (h_2 + h_3)^dagger chi_j for every
 * orbital j (Eqs. BITCSCF and BITCSCFconj without the one-body terms).
 * phi_R: right orbitals phi; phi_L: left orbitals chi; occ: host [Nk][nbands]
 * occupations f in [0, 1] (only the first nocc bands act as partners).
 * out_R / out_L may be NULL to skip that side. */
tc_status tc_apply(tc_ctx* ctx, const void* phi_R, const void* phi_L, const double* occ,
                   void* out_R, void* out_L, void* cuda_stream);

/* TC pseudo-energy per unit cell, both spins (Eqs. EtotTC / EtotBiTC with a
 * biorthonormal pair, single-determinant evaluation):
 * E = (2/Nk) Re sum_{k,mu} f [<chi|T|phi> + <chi|h_2 phi>/2 + <chi|h_3 phi>/3].
 * E_terms (nullable) receives the TC_NTERMS contributions.  Blocks the host. */
tc_status tc_energy(tc_ctx* ctx, const void* phi_R, const void* phi_L, const double* occ,
                    double* E_total, double* E_terms, void* cuda_stream);

/* Gradient of the energy of tc_energy (Eqs. EtotTC / EtotBiTC in the
 * single-determinant form given there).
 * Convention for the orbital gradients: g = dE/dRe(c) + i dE/dIm(c), so that
 * dE = Re sum conj(g) dc (PyTorch's convention for real functions of complex
 * tensors).  Layout as the orbitals.
 *   dE_dphiR  gradient with respect to the right orbitals phi  = (2/Nk) f (T chi + h^dagger chi)
 *   dE_dphiL  gradient with respect to the left orbitals chi   = (2/Nk) f (T phi + h phi)
 * i.e. the left and right operator outputs plus the kinetic term; this holds
 * with the SCF-mesh divergence corrections included.
 *   dE_dA[s], dE_dC[s]  partial derivatives with respect to A_s, C_s
 *   (s = 0 parallel, 1 antiparallel spins) at fixed orbitals.  E is a
 *   polynomial of degree 2 in the kernel data (Jastrow tables and correction
 *   coefficients), so each is the exact symmetric difference of two energy
 *   evaluations with the kernel data displaced along its derivative; the
 *   pair densities are recomputed in each evaluation.
 * Any output may be NULL (skipped).  Requires occ = 0 for bands >= nocc
 * (TC_ERR_ARG) and, for the orbital gradients, term_mask = 0
 * (TC_ERR_UNSUPPORTED).  Orbital outputs may be host or device pointers.
 * Blocks the host until the results are complete. */
tc_status tc_energy_grad(tc_ctx* ctx, const void* phi_R, const void* phi_L, const double* occ, void* dE_dphiR,
                         void* dE_dphiL, double dE_dA[2], double dE_dC[2], void* cuda_stream);

/* Biorthonormalises right and left orbitals in place, per k-point (Sec. 2.1:
 * <chi_i|phi_j> = delta_ij and <phi_i|phi_i> = 1; Sec. 2.3: Gram-Schmidt).
 * phi_R is orthonormalised by modified Gram-Schmidt in band order; phi_L is
 * replaced by chi_j = sum_i chi'_i (M^-1)_ij, M_ij = <phi_i|chi'_j> (FP64,
 * partial pivoting), which keeps the span of the left set.  All nbands bands
 * (at most 64).  Arrays may be host or device pointers; blocks the host.
 * TC_ERR_ARG if a norm or a pivot vanishes (outputs then undefined). */
tc_status tc_biorthonormalize(tc_ctx* ctx, void* phi_R, void* phi_L, void* cuda_stream);

/* One block-Davidson step for every k-point (Sec. 2.4), with a subspace of
 * two blocks (p_max = 1, the paper's default block count).  The operator is
 * h = T + the two- and three-body TC terms of tc_apply (right side) for the
 * partners given by the first nocc bands of (phi_R, phi_L, occ), which stay
 * fixed during the step; there is no pseudopotential.  Per k-point:
 *   v_i = phi_R band i (i < nbands; orthonormal per k on entry);
 *   w_i = P (h - eps_i) v_i, eps_i = <v_i|h|v_i>, Payne's preconditioner
 *         P(x) = (27+18x+12x^2+8x^3)/(27+18x+12x^2+8x^3+16x^4),
 *         x(G) = |k+G|^2/2 / <v_i|T|v_i> (P = 1 at |k+G| = 0 and 0 elsewhere
 *         when <v_i|T|v_i> = 0);
 *   each w_i orthogonalised against v and the w kept before it; kept if the
 *   remaining norm is >= 1e-8 (so the subspace dimension d lies in
 *   [nbands, 2 nbands]);
 *   M_ab = <b_a|h|b_b> over b = (v, kept w); its right and left eigenvectors
 *   y, z (z^H y = 1) for the nbands eigenvalues of lowest real part, in
 *   ascending order of the real part;
 *   phi_out_i = sum_a y_ai b_a, chi_out_i = sum_a z_ai b_a, then phi_out
 *   orthonormalised by Gram-Schmidt and chi_out made biorthonormal to it
 *   (as tc_biorthonormalize) -- the next step's trial vectors.
 * Arguments: phi_R, phi_L, phi_out, chi_out are orbital arrays (layout above;
 * host or device); the outputs must not alias the inputs or each other.
 * occ: host [Nk][nbands] in [0, 1] (only the first nocc bands act as
 * partners).  eig_out (optional): complex FP64 [Nk][nbands] Ritz values,
 * host or device.  dim_out (optional): int [Nk] subspace dimensions, host or
 * device.  The operator launches run in the context's precision; everything
 * else in FP64.  The first call allocates the step's buffers and a second
 * operator context with nocc + nbands bands (freed by tc_destroy).  At most 64
 * bands.  Blocks the host until the results are complete.  TC_ERR_NUMERIC if
 * the subspace eigen-solver does not converge or a Ritz vector set is
 * singular (outputs then undefined). */
tc_status tc_davidson_step(tc_ctx* ctx, const void* phi_R, const void* phi_L, const double* occ, void* phi_out,
                           void* chi_out, void* eig_out, int* dim_out, void* cuda_stream);

/* Crystal symmetry (Sec. 2.3 end, Sec. 2.6.4).  rot: nops integer 3x3
 * matrices S, row-major, acting on fractional real-space coordinates
 * (x -> S x; symmorphic operations, no translation); they must include the
 * identity, keep the lattice metric and map the k mesh onto itself.
 * time_reversal != 0 adds k -> -k.  The mesh points are taken in order; a
 * point that no earlier irreducible point reaches is irreducible, and its
 * images under the operations (then, with time reversal, the operations
 * times -1), in the given order, claim the points they reach first:
 * k = tr S^T k0 - K with tr = +-1 and K an integer vector (reciprocal
 * fractional coordinates).  From then on tc_apply / tc_energy /
 * tc_energy_grad / tc_davidson_step compute the occupied-pair stage
 * (Algs. 4, 6, 8, 11) for irreducible q2 only and obtain the other q2 by
 * rotation, and compute the outputs of irreducible k-points only, the others
 * following by the same unfolding as the orbitals.  This is exact when the
 * orbitals obey the symmetry (as tc_symmetrize_orbitals makes them); other
 * inputs give undefined results.
 * Needs the pair densities to fit the FFT box without wrapping (the Miller
 * span of all spheres, per axis, at most n/2 - 1), else TC_ERR_UNSUPPORTED.
 * nops = 0 switches the reduction off.  Synchronises the device and may
 * re-allocate the workspace (a different partner-chunk count).  Not for
 * batch contexts (TC_ERR_STATE). */
tc_status tc_set_symmetry(tc_ctx* ctx, int nops, const int* rot, int time_reversal);
/* Number of irreducible k-points and, if kmap6 is not NULL, per k-point
 * {k0, operation, tr, K1, K2, K3} (host int [Nk][6]); without symmetry every
 * point is its own (identity, tr = 1, K = 0). */
tc_status tc_symmetry_info(const tc_ctx* ctx, int* nirr, int* kmap6);
/* Overwrites the orbitals of every non-irreducible k-point (all bands, phi_R
 * and phi_L alike) by those of its irreducible point (Sec. 2.3):
 * c_k(tr S^T m0 + K) = c_k0(m0), conjugated when tr = -1.  Host or device
 * pointers; with host pointers the call returns after the copies. */
tc_status tc_symmetrize_orbitals(tc_ctx* ctx, void* phi_R, void* phi_L, void* cuda_stream);

/* Batched 3D FFT of `batch` contiguous n^3 complex volumes in place on the
 * device (precision TC_FP64: complex128, TC_FP32: complex64), sign -1
 * (sum f e^{-2 pi i m.r/n}) or +1; unnormalised.  Exposes the library's
 * shared-memory FFT for testing. */
tc_status tc_fft3d(int n, int precision, int sign, void* data, int batch, void* cuda_stream);

/* Device-time profiling of the stages of tc_apply / tc_energy.  Stage
 * indices: 0 orbitals to real space, 1 densities and Hartree-type fields,
 * 2 occupied-pair stage (Algs. 4, 6, 8, 11), 3 fused pair chains
 * (Algs. 2, 5, 6, 9, 11, 12), 4 the 3b4 pass (Alg. 10), 5 local terms,
 * corrections and sphere gather.  While enabled, each call records CUDA
 * events between stages on its stream and waits for them at its end; times
 * accumulate until tc_profile(ctx, 1) is called again. */
enum { TC_NSTAGES = 6 };
tc_status tc_profile(tc_ctx* ctx, int enable);
/* Autotuner of the partner-chunk counts: runs the operator on the given
 * inputs once per candidate count s = 1 .. min(8, Nk nocc) (after one
 * warm-up), for two-sided launches (tc_apply, tc_energy_grad) and then for
 * one-sided ones (tc_energy, tc_davidson_step), and keeps, separately for
 * each, the smallest s whose device time is within 2 % of the shortest for
 * the occupied-pair stage and for the pair-chain and 3b4 stages; so_out /
 * sc_out return the two-sided choices.  The chunk count changes only the order of partial sums (results
 * agree to rounding).  Orbital arrays host or device, occ host; resets the
 * per-stage times; re-allocates the workspace; blocks the host.  Not for
 * batch contexts (TC_ERR_STATE). */
tc_status tc_autotune(tc_ctx* ctx, const void* phi_R, const void* phi_L, const double* occ, int* so_out,
                      int* sc_out, void* cuda_stream);
/* ms[i] = accumulated device time of stage i (ms), launches[i] = kernel launches; n >= TC_NSTAGES. */
tc_status tc_stage_times(const tc_ctx* ctx, double* ms, int* launches, int n);
/* tc_pair_kernels -- which kernels the pair stages of this context's applies run (the fused pair
 * chains of Algs. 2, 5, 6, 9, 11, 12; the 3b4 pass of Alg. 10; the occupied-pair stage of Algs. 4,
 * 6, 8, 11).  For each of the three, in that order, info[3 i .. 3 i + 2] =
 *   kind:    0 full transforms, one CTA per item; 1 transforms pruned to the pair-density
 *            support, one CTA per item; 2 transforms on the support (or full) split over a
 *            thread-block cluster, the volumes in the CTAs' distributed shared memory
 *   support: transform points per axis on the spectral side (the box size n for full transforms)
 *   ctas:    CTAs per item (the cluster width; 1 for kinds 0 and 1)
 * The choice follows from the box size, the precision, the Miller span of the spheres (support
 * 2 span + 1) and whether the device can hold the kernel's cluster; every kind computes the same
 * operator.  info: 9 ints (host).  Errors: TC_ERR_STATE (null context, or a batch: ask its cells,
 * tc_batch_cell), TC_ERR_ARG (null info). */
tc_status tc_pair_kernels(const tc_ctx* ctx, int* info);

/* tc_pair_mirror -- whether two-sided applies of this context mirror their pair chains.  The left
 * operator (Eq. BITCSCFconj) of output q and partner j has the complex conjugate of the right pair
 * density of output j and partner q, and the kernel momentum -(k_j - k_q + G); with u~ real and
 * even (Appendix B) the left pair spectrum and the left antiparallel 3b6 spectrum of Alg. 12 are
 * the conjugate reflections (G -> -G) of the right ones.  A mirrored two-sided apply runs the right
 * pair chains first, storing those reflections for every pair whose output is itself a partner
 * (band < nocc), and the left chains then take them instead of recomputing them (7 of the 14
 * transforms of such a pair chain).  Exact up to rounding; used by TC_FP64 contexts whose pair
 * chains run the pruned kernels (tc_pair_kernels kind 1) on the SCF mesh without crystal symmetry,
 * with a buffer of (Nk nocc)^2 x 2 x support^3 complex FP64 values that tc_init allocates when it
 * fits in a quarter of the free device memory (not for FP32 contexts, whose pair chains are bound
 * by the loads that both sides keep; not for batch cells, band-point contexts or
 * tc_apply_noalloc).  *active = 1 when such a buffer is held (one-sided launches do not use it),
 * *bytes = its size (0 when inactive).  TC_FAULT=nomirror makes tc_init hold none, as if it did not
 * fit.  Either pointer may be NULL.  Errors: TC_ERR_STATE (null context or a batch). */
tc_status tc_pair_mirror(const tc_ctx* ctx, int* active, unsigned long long* bytes);

/* tc_band_constants -- the constants of the divergence corrections at
 * band-structure k-points off the SCF mesh (Sec. 2.6.3 after Eq.
 * divcorr_2ax_scf: Eqs. divcorr_2ax_band and 3b6_div_band1 use the scalar,
 * the grad-u band forms of Eq. correction_nabla the vector), with q over the
 * SCF mesh and alpha of params (0: the default):
 *   gamma_b[i]    = Omega/(4 sqrt(pi^3 alpha)) - (1/N_k) sum_{q,G} A_aux(k_i - q + G)
 *   W[3i .. 3i+2] = sum_{q,G} (k_i - q + G) A_aux(k_i - q + G)      (Cartesian, bohr)
 * A_aux(p) = exp(-alpha p^2)/p^2; 4 pi gamma_b/Omega equals minus the
 * Ewald-summed sum_{R != 0} cos(k.R)/|R| over the Born-von Karman supercell.
 * kfrac_band: [nkb][3] fractional coordinates in the reciprocal basis (host).
 * Host only, FP64, no device work (needs no GPU).  Errors: TC_ERR_ARG (null
 * pointer, nkb < 0, invalid params, a point on the SCF mesh modulo a
 * reciprocal vector: such a point takes the SCF constant Gamma0),
 * TC_ERR_UNSUPPORTED (box size); reason in tc_last_error(NULL). */
tc_status tc_band_constants(const tc_params* params, const double* kfrac_band, int nkb, double* gamma_b,
                            double* W);
/* tc_band_layout -- the plane-wave spheres of band-structure k-points (the
 * layout of orbitals at band points off the SCF mesh): for band point i,
 * npw[i] <- the number of Miller vectors m with |k_i + m.B|^2/2 <= ecut_ha,
 * and, if miller is not NULL, miller[i][g][3] <- those vectors in
 * lexicographic order (the order of every sphere of tc_layout), zero padded
 * to max_npw per point.  kfrac_band: [nkb][3] fractional coordinates (host);
 * call once with miller = NULL for the counts.  Host only, no device work.
 * Errors: TC_ERR_ARG (null pointer, nkb < 0, max_npw too small, a sphere that
 * does not fit the FFT box, invalid params), TC_ERR_UNSUPPORTED (box size). */
tc_status tc_band_layout(const tc_params* params, const double* kfrac_band, int nkb, int max_npw, int* npw,
                         int* miller);

/* tc_init_band / tc_apply_band -- the operator at band-structure k-points off the SCF mesh
 * (Sec. 2.6.3 after Eq. divcorr_2ax_scf; Sec. 2.6.4): output orbitals at nkb band points k_b,
 * partners on the SCF mesh.  Every partner-only field (densities, Hartree-type fields, the
 * occupied-pair stage with its 3a2 correction) is that of the SCF operator; the pair terms take
 * their kernels at k_b - q + G; the divergence corrections are the band forms: Eq.
 * divcorr_2ax_band and 3b6_div_band1/2/3 with Gamma_b, and the grad-u corrections of Eq.
 * correction_nabla with W(k_b) (Eqs. divcorr_2bx1/2, divcorr_3a3, div_corr_3b3_2,
 * div_corr_3a4_2/3, 3b5_div_2/3, div_corr_3b4_2/4), which use the band point's own occupied
 * orbitals (the first nocc band-point orbitals, occupations band_occ) and their occupied-pair fields
 * against the mesh partners (the constants are those of tc_band_constants).
 *
 * tc_init_band builds a context for params (the SCF mesh) and the band points kfrac_band
 * ([nkb][3] fractional coordinates, host; every point off the mesh modulo a reciprocal vector,
 * else TC_ERR_ARG).  Its tc_layout reports Nk + nkb k-points (the mesh, then the band points) and
 * one npw_max for all of them: every orbital array of tc_apply_band uses that npw_max.
 * tc_apply_band: phi_R, phi_L [Nk][nbands][npw_max] mesh orbitals (the partners, as tc_apply);
 * occ host [Nk][nbands]; band_phi_R, band_phi_L [nkb][nbands][npw_max] band-point orbitals on
 * their spheres (tc_band_layout order); band_occ host [nkb][nbands] (only the first nocc act, in
 * the corrections); out_R, out_L [nkb][nbands][npw_max] = (h_2 + h_3) phi_b and (h_2 + h_3)^dagger
 * chi_b at the band points (either may be NULL).  Device pointers only (TC_ERR_ARG otherwise); no
 * allocation; not thread-safe per context.  Other operator calls on a band context (tc_apply,
 * tc_energy, tc_energy_grad, tc_autotune, tc_biorthonormalize, tc_davidson_step, tc_set_symmetry)
 * return TC_ERR_STATE. */
tc_status tc_init_band(const tc_params* params, int nkb, const double* kfrac_band, tc_ctx** out);
tc_status tc_apply_band(tc_ctx* ctx, const void* phi_R, const void* phi_L, const double* occ, const void* band_phi_R,
                        const void* band_phi_L, const double* band_occ, void* out_R, void* out_L, void* cuda_stream);

/* tc_alu_peak -- measured fused multiply-add throughput of the current
 * device's non-tensor pipes, the denominator of the roofline of the FFT and
 * pair-product kernels (the paper has no counterpart: a measurement helper of
 * this library).  precision TC_FP32 or TC_FP64.  One launch of 16 independent
 * FMA chains per thread fills every SM; the iteration count doubles from a
 * short launch until one takes at least target_ms / 2 (0 < target_ms <=
 * 1000), then the fastest of three launches of that count gives
 * *tflops = 2 x FMAs / s / 1e12.  Runs on cuda_stream (NULL: legacy default
 * stream), blocks the host, allocates and frees a small output array.
 * Errors: TC_ERR_ARG (bad argument), TC_ERR_CUDA (reason in
 * tc_last_error(NULL)). */
tc_status tc_alu_peak(int precision, double target_ms, double* tflops, void* cuda_stream);

/* Size of the static device array behind tc_apply_noalloc: 64 MiB per device. */
#define TC_NOALLOC_MAX_BYTES 67108864

/* tc_apply_noalloc -- tc_apply for callers that cannot allocate device memory.
 * The paper has no counterpart: this is a convenience of this library.
 *
 * Who needs it: a host program whose framework has already reserved (almost)
 * all device memory for its own pool, so a cudaMalloc issued by this library
 * would fail, or one that forbids allocations from plug-in code during its
 * run.  Such a caller cannot use tc_init, which allocates the context's
 * tables and workspace.
 *
 * What it does: the same right and left operator as tc_apply (same arrays,
 * layouts, terms and term_mask), computed by the same kernels, for the
 * parameters given directly (no context).  Every device buffer of the call
 * is carved out of one file-scope device array of TC_NOALLOC_MAX_BYTES that
 * every GPU which has loaded the library holds until the process exits.  The
 * call makes no cudaMalloc, cudaFree or other allocating library call.  It
 * rebuilds the host setup (cell, spheres, kernel tables) on every call, so
 * it spends more host time than tc_apply with a reused context.
 *
 * Sizes: a problem whose buffers exceed TC_NOALLOC_MAX_BYTES is rejected with
 * TC_ERR_UNSUPPORTED before any device work; tc_last_error(NULL) states the
 * bytes it would need (a 16^3 box with 7 bands at one k-point in FP64 needs
 * about 30 MB).  Where the partner chunking that tc_init would choose (several
 * partial accumulators per orbital, for a fuller last wave of CTAs) does not
 * fit, the call runs with one chunk.
 *
 * Arguments: phi_R, phi_L, out_R, out_L must be device pointers (host
 * pointers give TC_ERR_ARG); out_R or out_L may be NULL to skip that side.
 * occ is a host array [Nk][nbands], read before the call returns.
 *
 * First call per device: it looks up the device address of the static array
 * (cudaGetSymbolAddress, with that device current) and sets the kernels'
 * shared-memory attributes and FFT twiddle constants.  With CUDA's lazy module
 * loading (the default since CUDA 12.2) the array's device memory is taken at
 * that moment, not when the library is loaded: make the first call on each
 * device before the host framework reserves its memory pool there, else it can
 * fail with TC_ERR_CUDA and a reason that names this.  With eager loading
 * (CUDA_MODULE_LOADING=EAGER) every device that loads the library holds the
 * array from then on, whether or not the entry point is called.
 *
 * Streams: every call uploads its tables and occupations from host memory
 * that lives only during the call, so it cannot be recorded into a CUDA graph;
 * a call on a stream that is capturing returns TC_ERR_STATE before any work.
 *
 * Sharing: all calls on a device use the same array, which keeps the
 * previous call's contents (each call clears what must start at zero).  Calls
 * whose GPU work overlaps -- on different streams, or from several threads
 * without ordering -- race on the array and give undefined results; order
 * them, e.g. on one stream.
 *
 * Errors: as tc_apply; the reason is given by tc_last_error(NULL). */
tc_status tc_apply_noalloc(const tc_params* params, const void* phi_R, const void* phi_L, const double* occ,
                           void* out_R, void* out_L, void* cuda_stream);

/* Batches of independent cells (many small problems of uneven size).
 *
 * tc_init_batch builds one context per cell (params[i]: each its own lattice,
 * k mesh, cutoff, box, bands and Jastrow; every cell the same precision) that
 * share one device workspace.  The workspace has L lanes, each as large as the
 * largest cell needs; cells are assigned to lanes by estimated cost (longest
 * first, least loaded lane), run one after another within a lane and
 * concurrently across lanes.  tc_apply_batch applies the operator (both sides,
 * as tc_apply) to every cell: the first call captures the whole schedule in a
 * CUDA graph.  To choose L it first times graphs for L = 1, 2, 4, 8, 16 (as
 * memory allows: a quarter of the free device memory) over a sample of at most
 * 12 cells spread over the cost order, and keeps the fastest; later calls
 * with the same arrays replay that graph with one launch on cuda_stream (new
 * arrays: one new capture).  Arguments are arrays of ncell pointers: device
 * orbital and output arrays in each cell's own layout, host occupations.
 * tc_apply_batch waits for the previous replay to finish before it returns
 * (the occupations are staged in pinned buffers); it does not wait for its own.
 *
 * tc_batch_cell returns cell i's context (owned by the batch: do not destroy
 * it) for tc_layout, tc_setup_scalars and single-cell calls; those use the
 * batch's workspace, so they must not overlap with a replay in flight.
 * tc_batch_info reports the number of cells, the chosen lane count (0 before
 * the first tc_apply_batch), the largest count memory allows, and the measured
 * replay time in ms of the tuning sample for L = 1, 2, 4, 8, 16 (-1 where not
 * tried).
 * tc_destroy on the batch frees every cell.  Single-cell entry points return
 * TC_ERR_STATE on a batch context. */
tc_status tc_init_batch(int ncell, const tc_params* params, tc_ctx** out);
tc_status tc_batch_cell(tc_ctx* batch, int i, tc_ctx** cell);
tc_status tc_apply_batch(tc_ctx* batch, const void* const* phi_R, const void* const* phi_L, const double* const* occ,
                         void* const* out_R, void* const* out_L, void* cuda_stream);
tc_status tc_batch_info(const tc_ctx* batch, int* ncell, int* lanes, int* lanes_max, double* tune_ms);

/* Reason of the last failure on ctx; with ctx == NULL, of the last failed
 * tc_init on the calling thread.  The string lives until the next call. */
const char* tc_last_error(const tc_ctx* ctx);
tc_status tc_destroy(tc_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* TC_GB300_H */
