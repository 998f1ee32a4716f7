/*
 * rttddft.h -- C ABI of the GB300 velocity-gauge RT-TDDFT step in an
 * auxiliary subspace (arXiv 2403.04351, Sec. 2).
 *
 * The problem (Sec. 2, Eq. evolution_wf_coeff): evolve the coefficient
 * matrices C_k (N_basis x N_states per k-point) of an LAPW+LO expansion
 * (Eq. expansion_LAPW_lo) under S_k dC_k/dt = -i H_k(t) C_k with the
 * velocity-gauge Hamiltonian H(t) = 1/2 (-i nabla + A(t)/c)^2 + V(r, t),
 * i.e. in the basis H(t) = H0 + (A/c).P + |A|^2/(2c^2) S + dV(t).
 * H and S are never formed: they act through the per-atom muffin-tin
 * blocks mapped by the matching coefficients A_alpha and the interstitial
 * table V~_{G-G'} (Eq. v_MT, Eq. v_interstitial, Appendix A).  The state is
 * carried in the auxiliary subspace of ground-state vectors CC(0)
 * (Eq. auxiliary_basis, approximation_coefficients): theta = CC^H S C,
 * d theta/dt = -i HH(t) theta with HH = CC^H H(t) CC
 * (Eq. evolution_of_projection_coeff, auxiliary_hamiltonian_with_parts).
 *
 * Conventions for every array argument unless stated otherwise:
 *  - complex numbers are interleaved pairs of doubles (re, im);
 *  - matrices are column-major with leading dimension = number of rows;
 *  - per-k arrays are concatenated over k in k order, per-atom arrays in
 *    atom order;
 *  - basis rows of a k-point are [N_G plane waves ; local orbitals], the
 *    local orbitals grouped by atom in atom order;
 *  - "host" pointers are ordinary CPU memory, read or written before the
 *    call returns; "host or device" pointers are classified with
 *    cudaPointerGetAttributes and device ones are read on the context's
 *    stream;
 *  - the caller owns every pointer it passes; the library copies what it
 *    keeps.  The context owns all device memory it allocates until
 *    rttddft_destroy.
 *
 * Errors: every int-returning call returns RTTDDFT_OK (0) or a negative
 * code below; rttddft_last_error gives a one-line description.  A call
 * that fails leaves the context usable unless it returned
 * RTTDDFT_ERR_CUDA.  Calls on one context are not thread-safe; calls on
 * different contexts are independent.  All device work is ordered on the
 * stream given at set-up.
 */
#ifndef RTTDDFT_H
#define RTTDDFT_H

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define RTTDDFT_API __attribute__((visibility("default")))
#else
#define RTTDDFT_API
#endif

#define RTTDDFT_OK 0
#define RTTDDFT_ERR_ARG (-1)             /* bad size, NULL or inconsistent argument */
#define RTTDDFT_ERR_NOT_HERMITIAN (-2)   /* h, o, p, dh or a V~ table not Hermitian */
#define RTTDDFT_ERR_NOT_PD (-3)          /* o_alpha or the trial overlap not positive definite */
#define RTTDDFT_ERR_NOT_ORTHONORMAL (-4) /* given CC(0) not S-orthonormal */
#define RTTDDFT_ERR_NONFINITE (-5)       /* NaN or Inf in an input */
#define RTTDDFT_ERR_OOM (-6)             /* device allocation failed */
#define RTTDDFT_ERR_CUDA (-7)            /* a CUDA call failed */
#define RTTDDFT_ERR_TIMEOUT (-8)         /* an iteration limit on the device ran out */
#define RTTDDFT_ERR_UNSUPPORTED (-9)     /* option value not built */

/* propagator for Eq. evolution_of_projection_coeff over one step dt,
 * with HH held at the step midpoint value A_k = A(t_k + dt/2) */
#define RTTDDFT_PROP_CHEBYSHEV 0 /* exp(-i HH dt) by its Chebyshev series, truncated at FP64 round-off */
#define RTTDDFT_PROP_EIG 1       /* exp(-i HH dt) = V e^{-i Lambda dt} V^H from a Jacobi eigensolver */
#define RTTDDFT_PROP_CN 2        /* Crank-Nicolson (I + i dt/2 HH)^{-1} (I - i dt/2 HH), by its Chebyshev series */

/* precision of the full-basis contractions (expand, operator, project);
 * the subspace propagation and every reduction stay FP64 */
#define RTTDDFT_PREC_FP64 0
#define RTTDDFT_PREC_FP32 1
/* split-BF16 on the tensor cores: the interstitial convolution and the
 * matching-coefficient products of the operator run as tcgen05 products of
 * bf16 hi/lo splits (hi.hi + hi.lo + lo.hi, FP32 accumulation, the K slices
 * summed as FP32 two-sum pairs into FP64, relative error a few 2^-16); the
 * muffin-tin blocks too when there are 16 to 64 states; the other full-basis
 * contractions as in RTTDDFT_PREC_FP32.  At most 128 states. */
#define RTTDDFT_PREC_BF16X3 2
/* split-FP16: the same products with fp16 hi/lo splits (22 significant bits,
 * relative error a few 2^-22): the matching coefficients and the V~ table are
 * scaled by powers of two so that their largest entry sits near 2^14 (the
 * per-step table V~ + s dV~ may reach 4 times the largest |V~|), C by 2^12
 * (|c| <= 16) and [hQ | oQ] by 2^10 (<= 64); a scaled value outside the fp16
 * range makes the step fail with ERR_NONFINITE.  At most 128 states. */
#define RTTDDFT_PREC_FP16X3 3

/* how the interstitial sum of Eq. v_interstitial, sum_G' V~_{G-G'} C_G', is
 * evaluated (Sec. 3: matrix products against FFTs) */
#define RTTDDFT_INTERSTITIAL_TOEPLITZ 0 /* direct sum over G' with V~_{G-G'} generated from the table */
/* circular convolution on a grid of F_i >= vt_dim[i] points per axis (the
 * smallest products of 2, 3 and 5, at most 512): pruned inverse and forward
 * 3-D FFTs around a product with the table's real-space image, FP64 in the
 * FP64 form and FP32 in the others (the split forms keep the matching-
 * coefficient products on the tensor cores); ERR_UNSUPPORTED when an axis
 * needs more than 512 points, ERR_OOM when the transform buffers (N_aux
 * columns of the planes holding a G, per k-point) do not fit.  Equal to the
 * direct sum up to rounding. */
#define RTTDDFT_INTERSTITIAL_FFT 1

/* how the auxiliary basis CC(0) is obtained at set-up */
#define RTTDDFT_AUX_RITZ 0  /* Ritz vectors of H0 in span(caux): S-orthonormal, H0-diagonal */
#define RTTDDFT_AUX_GIVEN 1 /* caux and eps used as given; S-orthonormality is checked */

typedef struct rttddft_ctx rttddft_ctx;

/* The synthetic or physical system (all host pointers, read during set-up). */
typedef struct {
    int n_k;            /* number of k-points, >= 1 */
    int n_atoms;        /* number of atoms (muffin-tin spheres), >= 0 */
    int n_s;            /* N_states propagated per k-point, 1 <= n_s <= n_aux */
    int n_aux;          /* N_aux, auxiliary subspace dimension, <= N_basis of every k */
    double omega;       /* unit-cell volume (bohr^3), > 0 */
    double c_light;     /* speed of light (a.u.), > 0 */
    const double* occ;  /* [n_s] occupations f_j */
    const double* wk;   /* [n_k] k-point weights */
    const int* n_g;     /* [n_k] plane waves N_G per k-point */
    const int* g_int;   /* [sum n_g][3] integer G triples, row-major */
    const double* gk;   /* [sum n_g][3] cartesian G+k (1/bohr), row-major */
    const int* n_a;     /* [n_atoms] matching rows N_A per atom */
    const int* n_lo;    /* [n_atoms] local orbitals per atom */
    const double* amat; /* complex; per k: (sum n_a) x n_g[k] matching coefficients,
                           atoms stacked along the rows (Eq. v_MT's A_k) */
    const double* h;    /* complex; per atom m x m, m = n_a + n_lo: H0 muffin-tin block
                           [V_LL V_Ll; V_lL V_ll] of Eq. v_MT (Hermitian) */
    const double* o;    /* complex; per atom m x m overlap block (Hermitian positive definite) */
    const double* p;    /* complex; per atom 3 consecutive m x m momentum blocks (x, y, z) */
    int vt_dim[3];      /* odd extents of the interstitial table box */
    const double* vtab; /* complex; V~_g for g_i in [-(vt_dim[i]-1)/2, (vt_dim[i]-1)/2],
                           row-major over (g_0, g_1, g_2), last index fastest; Hermitian in g */
    const double* caux; /* complex; per k: N_basis x n_aux; trial vectors (RITZ) or CC(0) (GIVEN) */
    const double* eps;  /* [n_k][n_aux] eigenvalues for GIVEN mode; NULL for RITZ */
    const double* c0;   /* complex; NULL (C(0) = first n_s columns of CC(0)) or per k N_basis x n_s */
    double recip[9];    /* reciprocal lattice vectors b_1, b_2, b_3 (rows, 1/bohr): G = n_1 b_1 + n_2 b_2 + n_3 b_3;
                           needed by the Hartree feedback only (zeros otherwise) */
} rttddft_system;

typedef struct {
    double dt;          /* time step (a.u.), > 0 */
    int propagator;     /* RTTDDFT_PROP_* */
    int precision;      /* RTTDDFT_PREC_* */
    int reproject;      /* 0: carry theta; 1: theta <- Lowdin-orthonormalised CC^H S C each step (FP64 only) */
    int aux_mode;       /* RTTDDFT_AUX_* */
    int max_record;     /* capacity of the per-step observable record, >= 1 */
    int graph_steps;    /* steps per captured CUDA graph (>= 1); 0 launches kernels directly */
    double cheb_tol;    /* truncation of the Chebyshev series (default 1e-16) */
    double ortho_tol;   /* GIVEN mode: max |CC^H S CC - I| accepted (default 1e-10) */
    int max_sweeps;     /* iteration limit of the Jacobi eigensolver (default 30) */
    double a_max;       /* bound on |A(t)| used for the Chebyshev spectral interval; 0: taken
                           from the samples of each call (device samples are then read back) */
    double s_max;       /* bound on |s_k| of the potential change; 0: from the samples */
    int interstitial;   /* RTTDDFT_INTERSTITIAL_* (default TOEPLITZ) */
    /* 1: the potential change of every step is the Hartree potential of the interstitial density's
     * change since the start, dV_g = 4 pi (n_g(t_k) - n_g(0)) / |g|^2 on the table box (g != 0),
     * n_g = (1/Omega) sum_k w_k sum_j f_j sum_G C_Gj conj(C_(G-g)j) from the plane-wave rows of C_k;
     * it enters HH and the operator of step k (Sec. 2: VV(t) is the part rebuilt every step).
     * Needs the FFT route and recip; rttddft_set_dv and dv_scale are then refused (ERR_ARG), the
     * adjoint is not built (ERR_UNSUPPORTED).  Default 0. */
    int hartree;
    double hartree_bound; /* bound on sum_g |dV_g| >= ||dVV||_2 used for the Chebyshev interval; a step whose
                             change exceeds it fails with ERR_ARG (default 0.1 Ha) */
    /* with hartree = 1: the muffin-tin part of the feedback.  0 (default): none.  U != 0: per atom the
     * density matrix of its matching and local-orbital channels, n_a = sum_k w_k sum_j f_j (E_a c_j)(E_a c_j)^H
     * with E_a = [A_a 0; 0 I] (Appendix A), taken in FP64 from theta through the atom's rows of E_a CC, and
     * the on-site blocks dh_a = U (n_a(t_k) - n_a(0)) act like the dh of rttddft_set_dv with s = 1 (the
     * radial functions that would turn n_a into a potential are not part of this interface; the contact
     * form stands in for them).  The bound above then covers sum_g |dV_g| + sum_a ||dh_a||_F max_k ||L_ka||_F^2
     * (L_ka the atom's rows of E_a CC at k-point k). */
    double hartree_mt_u;
} rttddft_options;

/* Per-step records (all k-points summed with their weights), caller-allocated
 * host arrays of `capacity` records.  Record r belongs to time t[r] = t_(r+1). */
typedef struct {
    int capacity;       /* in: records the arrays can hold */
    int count;          /* out: records written */
    double* t;          /* [capacity] time after the step */
    double* j;          /* [capacity][3] J = -(1/Omega) sum w f Re theta^H (PP + A/c SS) theta */
    double* j_full;     /* [capacity][3] the same from the full-basis C via the operator pass */
    double* dmu;        /* [capacity][3] delta mu = Omega int J_ind dt (Eq. dipole, trapezoid) */
    double* energy;     /* [capacity] sum w f Re c^H H(A_k) c */
    double* norm_dev;   /* [capacity] max |C^H S C - I| over k */
    double* resid;      /* [capacity] max |CC^H S C - theta| over k */
    double* dt_cr;      /* [capacity] f/(lambda_max - lambda_min) of HH (Eq. critical_timestep, f = 0.2);
                           spectral bounds for the Chebyshev forms, eigenvalues for EIG */
    double* n_exc;      /* [capacity] or NULL: excited electrons N_e - sum w f sum_{i < N_s} |theta_ij|^2,
                           the charge that left the N_s lowest auxiliary vectors (the occupied
                           ground state when C(0) is the default) */
} rttddft_obs;

typedef struct {
    long long steps_done;  /* steps taken since set-up */
    double time;           /* t after the last step */
    int n_basis_max;       /* largest N_basis over k */
    int cheb_terms;        /* terms of the last Chebyshev series */
    double dt_cr0;         /* Eq. critical_timestep from the set-up eigenvalues, min over k */
    int kernel_launches_per_step; /* kernels launched per step (graph nodes) */
    int precision;         /* RTTDDFT_PREC_* of the context */
    int tc_tile_n;         /* split-BF16 form: real output columns per tensor-core tile (0 otherwise) */
    int tc_stages;         /*   100 x generated-operand stages + copied-operand stages */
    int tc_kblocks;        /*   K blocks (32 G') per slice */
    int tc_slices;         /*   K slices */
    int tc_window;         /*   largest interstitial table window staged (entries) */
    int tc_smem;           /*   dynamic shared memory per block (bytes) */
    int tc_candidates;     /*   launch shapes timed by the set-up autotuner */
    int tc_interstitial_ns;/*   tuned time of the interstitial launch (ns) */
    int tc_matching_ns;    /*   tuned time of the matching-row launch (ns) */
    int interstitial;      /* RTTDDFT_INTERSTITIAL_* of the context */
    int fft_grid[3];       /* FFT route: grid points per axis (0 otherwise) */
    int fft_fused;         /*   1: a plane's two in-plane axes in one launch (chosen at set-up by timing) */
    int tc_gen_threads;    /* split forms: threads generating the interstitial operand per block (256 or 512) */
    int tc_a_tmem;         /*   1: that operand is written to tensor memory (0: shared memory) */
    int tc_back_parts;     /*   back-projection launched in 1 or 2 output-column parts (0: none) */
} rttddft_info;

RTTDDFT_API void rttddft_default_options(rttddft_options* opt);

/* Validate `sys`, copy it to the device, build the auxiliary basis and the
 * projected momentum PP = CC^H P CC (Eq. auxiliary_hamiltonian_with_parts),
 * and set theta(0).  `cuda_stream` is a cudaStream_t (NULL: legacy default
 * stream).  On success *out owns the device state.
 * Errors: ERR_ARG, ERR_NOT_HERMITIAN, ERR_NOT_PD (o_alpha, or a rank-deficient
 * trial block), ERR_NOT_ORTHONORMAL (GIVEN), ERR_NONFINITE, ERR_OOM,
 * ERR_CUDA, ERR_UNSUPPORTED, ERR_TIMEOUT (Jacobi sweep limit). */
RTTDDFT_API int rttddft_setup(const rttddft_system* sys, const rttddft_options* opt, void* cuda_stream,
                  rttddft_ctx** out);

/* Advance every k-point by `nsteps` steps (Sec. 2): build HH(t_k), propagate
 * theta, expand C = CC theta (Eq. approximation_coefficients), apply H(t)
 * and S to C from the submatrices, project CC^H S C, and reduce J, dmu and
 * E into the record.  a_samples: host or device, [nsteps][3], A on
 * [t_k, t_k + dt) (the midpoint value).  dv_scale: NULL, or host or device
 * [nsteps] scales s_k of the potential change set by rttddft_set_dv.
 * The call returns once the work is enqueued on the context's stream (host
 * samples are staged through pinned memory first); it waits for the device
 * only when device samples must be read back (a_max or s_max left at 0) or
 * when a wider spectral interval is needed.  |A_k| above a nonzero a_max
 * (or |s_k| above s_max) is ERR_ARG for host samples; for device samples it
 * is detected on the device and reported by the next call.  A Jacobi
 * iteration limit that ran out (EIG propagator) is reported as ERR_TIMEOUT by
 * the next call that waits for the device (observables, get_state, step).
 * Errors: ERR_ARG (nsteps < 1, the record would overflow, a bound exceeded),
 * ERR_NONFINITE (host samples), ERR_CUDA, ERR_TIMEOUT. */
RTTDDFT_API int rttddft_step(rttddft_ctx* ctx, int nsteps, const double* a_samples, const double* dv_scale);

/* Copy the records out (host arrays, see rttddft_obs); clear != 0 empties
 * the record afterwards.  Error: ERR_ARG if out->capacity < the records held. */
RTTDDFT_API int rttddft_observables(rttddft_ctx* ctx, rttddft_obs* out, int clear);

/* Set the potential-change pattern dV_1 (Appendix A): dh complex, per atom
 * m x m Hermitian muffin-tin blocks concatenated; dvtab complex, same box as
 * vtab, Hermitian in g.  Host pointers.  Steps given a dv_scale array then
 * use dV(t_k) = s_k dV_1 in H(t) and rebuild dHH = CC^H dV(t_k) CC every
 * step from the scaled blocks (Eq. v_MT, Eq. v_interstitial).
 * Errors: ERR_ARG, ERR_NOT_HERMITIAN, ERR_NONFINITE, ERR_CUDA. */
RTTDDFT_API int rttddft_set_dv(rttddft_ctx* ctx, const double* dh, const double* dvtab);

/* Apply the operator from submatrices (Eq. v_MT, Appendix A) to an N_basis x
 * ncols block X of k-point k: HX = H(A) X (+ s dV_1 X) and SX = S X.
 * x, hx, sx: host or device (all three of the same kind), complex,
 * column-major with leading dimension N_basis(k).  a_vec: host [3].
 * Errors: ERR_ARG, ERR_CUDA, ERR_OOM. */
RTTDDFT_API int rttddft_apply(rttddft_ctx* ctx, int k, int ncols, const double* x, const double* a_vec,
                  double dv_scale, double* hx, double* sx);

/* The same operator as rttddft_apply, for callers that must not allocate
 * device memory at the time of the call (a CUDA graph being captured, an
 * allocator-free thread, memory owned by another pool).  The paper has no
 * counterpart; this is a property of the library, not of the method.
 * x, hx, sx must be device pointers (complex, N_basis(k) x ncols,
 * column-major); the call is asynchronous on the context's stream and does
 * not wait for the device.  Its scratch is one 16 MiB array in device memory
 * that every GPU loading the library holds until the process exits; the
 * first call on each device looks up that array's address (make that first
 * call before starting any stream capture).  Every call shares the array, so
 * calls whose work overlaps on the GPU (different streams or contexts) race;
 * calls on one stream are ordered.  The scratch need of a k-point is, in
 * bytes, 48 N_basis N_states (the staged block and [HX | SX]) + 48 M_A N_states
 * (Q = A X and the muffin-tin products, M_A = matching rows of all atoms)
 * + 16 M_A N_states ceil(N_G / K_chunk) (split-K partials of Q) + the
 * interstitial partials of the direct sum, 32 n_slot n_tsel max_k N_G
 * (n_slot row segments of the table window, n_tsel column groups; these
 * dominate) + 16 bytes per V~ table entry when dv_scale != 0 (24 in the
 * reduced-precision forms) + a few small per-row sums, each part rounded up
 * to 256 bytes.
 * Among the benchmark's workloads tiny400 (N_basis 400) fits and co_12000
 * (N_basis 12000, N_states 7) does not; a k-point that does not fit is
 * rejected with ERR_ARG and a message giving its need.  The caller's current
 * device must be the one the context was set up on (ERR_ARG otherwise).
 * It never calls cudaMalloc or cudaFree.
 * Errors: ERR_ARG (bad sizes, NULL or host pointers, scratch limit, another
 * current device), ERR_CUDA, ERR_UNSUPPORTED (device ordinal above 255). */
RTTDDFT_API int rttddft_apply_noalloc(rttddft_ctx* ctx, int k, int ncols, const double* x,
                                      const double* a_vec, double dv_scale, double* hx, double* sx);

/* State of k-point k.  theta: complex n_aux x n_s; c: NULL or complex
 * N_basis(k) x n_s (the last expanded C).  Host pointers. */
RTTDDFT_API int rttddft_get_state(rttddft_ctx* ctx, int k, double* theta, double* c);
RTTDDFT_API int rttddft_set_state(rttddft_ctx* ctx, int k, const double* theta);

/* Auxiliary basis of k-point k after set-up: caux complex N_basis(k) x n_aux,
 * eps [n_aux] ascending, pp complex 3 x n_aux x n_aux (may be NULL).  Host. */
RTTDDFT_API int rttddft_get_aux(rttddft_ctx* ctx, int k, double* caux, double* eps, double* pp);

RTTDDFT_API int rttddft_get_info(rttddft_ctx* ctx, rttddft_info* info);

/* Gradient of gdir . [dmu(t0 + nsteps dt) - dmu(t0)] with respect to every
 * pulse sample A_k (k < nsteps, 3 components), where t0 is the context's
 * current time: reverse mode through the propagated steps (the exact
 * adjoint of the computed Chebyshev polynomial), theta checkpointed every
 * `ckpt_every` steps and recomputed per segment.  The context's state,
 * time and records are left unchanged.  a_samples, dv_scale: as for
 * rttddft_step; gdir host [3]; grad host [nsteps][3]; dmu_out NULL or host [3]
 * (the dipole increment of the forward pass).  Requires the Chebyshev
 * propagator.  Errors: ERR_ARG, ERR_UNSUPPORTED, ERR_OOM, ERR_CUDA. */
RTTDDFT_API int rttddft_adjoint(rttddft_ctx* ctx, int nsteps, const double* a_samples, const double* dv_scale,
                    const double* gdir, int ckpt_every, double* grad, double* dmu_out);

/* Per-kernel timing of the step: runs `nsteps` steps exactly as rttddft_step
 * does, but with kernels launched one by one (no graph) and a CUDA event
 * recorded on the context's stream after each launch.  out->names[i] (static
 * strings owned by the library) and out->ms[i] (device milliseconds summed
 * over the steps) describe the i-th launch slot of a step; out->count slots
 * are filled, at most out->capacity.  The steps advance the state and the
 * record like rttddft_step.  a_samples, dv_scale: host arrays.
 * Errors: ERR_ARG, ERR_CUDA. */
typedef struct {
    int capacity;        /* in: slots the arrays hold */
    int count;           /* out: launch slots per step */
    const char** names;  /* [capacity] out */
    double* ms;          /* [capacity] out, summed over the steps */
} rttddft_trace;
RTTDDFT_API int rttddft_trace_steps(rttddft_ctx* ctx, int nsteps, const double* a_samples,
                                    const double* dv_scale, rttddft_trace* out);

/* Dynamical polarizability (Eq. polarizability) from a recorded time series:
 *   alpha_{l l'}(w) = (i Omega / w) J_l(w) / E_l'(w),
 *   F(w) = dt sum_{n < n_t} f(t_n) e^{(i w - eta) t_n},  t_n = t0 + n dt,
 * for f = the induced current J_ind = J - J(t0) (e.g. the record's j minus its
 * field-free value) and f = the electric field E = -(1/c) dA/dt at the same
 * times; eta >= 0 damps the finite window.  One GPU block per frequency, FP64
 * sums in a fixed order.
 *   j_ind, e_field  [n_t][3] (host or device);  w [n_w] frequencies > 0 (host or
 *                   device; host values are checked);  omega_cell = Omega > 0;
 *   out_j, out_e    [n_w][3] complex J(w), E(w), or NULL;
 *   alpha           [n_w][3][3] complex, row l, column l' (l' fastest), or NULL;
 *                   an entry with E_l'(w) exactly zero is written as 0.
 * Each output pointer may be host or device memory (classified like the inputs);
 * the call returns after the results are written.  Errors: ERR_ARG (sizes, dt <= 0, a host w <= 0, NULL
 * inputs), ERR_CUDA. */
RTTDDFT_API int rttddft_polarizability(int n_t, double t0, double dt, const double* j_ind, const double* e_field,
                                       double eta, int n_w, const double* w, double omega_cell, double* out_j,
                                       double* out_e, double* alpha, void* cuda_stream);

/* Split-BF16 complex GEMM on the tensor cores, the contraction form of the
 * precision option RTTDDFT_PREC_BF16X3 (the bulk contractions of Sec. 2:
 * expansion C = CC theta, Eq. approximation_coefficients, and projection
 * CC^H S C, Eq. evolution_of_projection_coeff):
 *   C = op(A) X          (beta_add = 0)   or   C += op(A) X  (beta_add = 1),
 * op(A) = A (trans = 0, A is m x k) or A^H (trans = 1, A is k x m); X is
 * k x n; C is m x n.  The complex product is one real GEMM on
 * [Re A | Im A] and, per column of X, [Re x | -Im x] and [Im x | Re x]; each
 * real operand is split as v = hi + lo with hi, lo bf16, and
 * hi.hi + hi.lo + lo.hi is accumulated in FP32 on the tensor cores per slice
 * of K, the slices summed in FP64.  Error per element: a few 2^-16 of
 * sum_k |a||x| (the dropped lo.lo term and the rounding of lo).
 * a, x, c: device pointers, complex, column-major, lda >= rows of A,
 * ldx >= k, ldc >= m.  stream: a cudaStream_t or NULL.  The call allocates
 * and frees its own workspace (about (m + 2n) x 8k bytes) and synchronizes
 * the stream before it returns.  m, n or k = 0 is allowed (C unchanged for
 * k = 0 with beta_add = 1, zero otherwise).
 * Errors: ERR_ARG (sizes, leading dimensions, NULL), ERR_OOM, ERR_CUDA,
 * ERR_TIMEOUT (a bounded wait of the copy/product pipeline ran out),
 * ERR_UNSUPPORTED (the driver has no tensor-map encoder). */
RTTDDFT_API int rttddft_zgemm_bf16x3(int trans, int m, int n, int k, const double* a, int lda, const double* x,
                                     int ldx, double* c, int ldc, int beta_add, void* stream);

RTTDDFT_API void rttddft_destroy(rttddft_ctx* ctx);

/* Text of the last error on `ctx` (or of the last failed rttddft_setup in
 * this thread when ctx is NULL).  The string lives until the next call. */
RTTDDFT_API const char* rttddft_last_error(const rttddft_ctx* ctx);

RTTDDFT_API const char* rttddft_version(void);

#ifdef __cplusplus
}
#endif
#endif /* RTTDDFT_H */
