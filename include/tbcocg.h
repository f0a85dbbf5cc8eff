/*
 * tbcocg.h -- C ABI of the GB300 generalized shifted COCG library.
 *
 * The library solves, for many complex energies z_k and unit right-hand
 * sides e_j, the linear systems of Eq. (base-2) in a non-orthogonal local
 * basis,
 *
 *     (z_k S - H) x_j(z_k) = e_j ,
 *
 * and returns the Green's-function elements G_ij(z_k) = (x_j(z_k))_i of
 * Eq. (GreensFunc), or their energy integral folded into Mulliken
 * populations.  H is the tight-binding Hamiltonian matrix and S the overlap
 * matrix of Section 2.2; both are real symmetric, S positive definite.
 * The solver is the generalized shifted COCG method of Section 3.3: one seed
 * system (Eq. shift-E) iterated by Eqs. (CGp:p), (CGp:x), (CGp:r) with
 * r' = S^-1 r from an inner solve (CG in FP64; with TB_MIXED, FP64
 * iterative refinement with FP32 corrections), every other shift carried by the scalar
 * recurrence Eq. (shift:pi) through the collinear residuals of
 * Eq. (collinear), and seed switching.  The generalized Lanczos process of
 * Section 3.2 (Eqs. 1.13, 1.18) is exported as well.
 *
 * Conventions for every entry point
 *  - Return value: tb_status, TB_OK = 0.  tb_status_string() names it.
 *  - Pointers are owned by the caller and are only read/written during the
 *    call; nothing is retained after it returns except inside a tb_handle.
 *  - Input arrays marked "host" are read on the host.  Output arrays marked
 *    "host or device" may be either: the library asks the CUDA runtime where
 *    the pointer lives and copies the result there.  Device outputs are
 *    complete when the call returns (the call synchronises the stream).
 *  - Complex numbers are pairs of doubles (real, imaginary), interleaved.
 *  - Orbital indices are in the caller's orbital order: the orbitals of atom
 *    0 first (s, then px, py, pz for sp atoms), then atom 1, and so on.
 *  - `stream` is a cudaStream_t passed as void*; NULL is the legacy default
 *    stream.  All device work of a call is enqueued on it.
 *  - Only one call may use a given handle at a time.
 *  - Shifts: 1 <= K <= 1024 finite complex z_k (and opts->seed < K), else
 *    TB_ERR_INVALID_ARG.  Im z_k != 0 keeps z_k S - H nonsingular (S is
 *    positive definite, H real symmetric); a real shift at or near an
 *    eigenvalue ends in TB_ERR_BREAKDOWN or TB_ERR_NOT_CONVERGED.
 *  - Columns: 1 <= R, every cols[c] in [0, N) (repeats allowed), else
 *    TB_ERR_INVALID_ARG; columns are solved in panels of opts->panel
 *    (a power of two <= 256; 0 picks one), a ragged last panel padded with
 *    inactive columns.
 */
#ifndef TBCOCG_H
#define TBCOCG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tb_handle tb_handle;

typedef enum {
    TB_OK = 0,
    TB_ERR_INVALID_ARG = 1,    /* malformed argument or block structure   */
    TB_ERR_NOT_SYMMETRIC = 2,  /* S or H (or their pattern) not symmetric */
    TB_ERR_S_NOT_SPD = 3,      /* S not positive definite (seen by CG)    */
    TB_ERR_OOM = 4,            /* device allocation failed                */
    TB_ERR_CUDA = 5,           /* a CUDA runtime call failed              */
    TB_ERR_NOT_CONVERGED = 6,  /* max_iter reached; converged shifts valid*/
    TB_ERR_BREAKDOWN = 7,      /* COCG breakdown (rho or mu == 0)         */
    TB_ERR_TIMEOUT = 8,        /* reserved: no kernel of this library waits
                                  on another CTA, flag or stream (grid
                                  reductions take arrival tickets and never
                                  spin), so no call returns it              */
    TB_ERR_NO_DEVICE = 9,      /* no usable CUDA device                   */
    TB_ERR_TOO_LARGE = 10      /* request exceeds the fixed scratch of the
                                  allocation-free entry point              */
} tb_status;

enum { TB_FP64 = 0, TB_MIXED = 1 };

/*
 * Block-sparse system in atom blocks (Section 2.2: one block per pair of
 * atoms within the overlap cutoff).  Block row i holds the blocks
 * bcol[brow_ptr[i]] ... bcol[brow_ptr[i+1]-1], sorted ascending, the
 * diagonal block included; the pattern holds both triangles and must be
 * symmetric.  Block (i, j) has orb_per_atom[i] x orb_per_atom[j] values,
 * row-major; the blocks are concatenated in block order.
 *
 * H_vals == NULL builds H by the ASED rule (Section 2.2, Eq. Hap-1) on the
 * device: H_{ia,ia} = eps_{ia}; H_{ia,ib} = 0 for a != b on one atom;
 * H_{ia,jb} = K (eps_{ia} + eps_{jb}) / 2 * S_{ia,jb} for i != j.
 * All arrays are host memory and are copied during tb_create.
 */
typedef struct {
    int32_t n_atoms;
    const int32_t *orb_per_atom; /* [n_atoms], 1 (s) or 4 (s,px,py,pz)  */
    const int64_t *brow_ptr;     /* [n_atoms+1]                          */
    const int32_t *bcol;         /* [nb]                                 */
    const double *S_vals;        /* concatenated blocks of S             */
    const double *H_vals;        /* concatenated blocks of H, or NULL    */
    const double *eps;           /* [N] on-site levels (eV); needed when
                                    H_vals == NULL, else may be NULL     */
    double K;                    /* ASED constant of Eq. Hap-1           */
    int32_t precision;           /* TB_FP64 (the handle serves both
                                    solve precisions)                    */
} tb_system_desc;

/* Validate the system, copy it to the device (H built by Eq. Hap-1 if not
 * given) and return a handle.  Errors: TB_ERR_INVALID_ARG (structure),
 * TB_ERR_NOT_SYMMETRIC (pattern or values), TB_ERR_OOM, TB_ERR_CUDA,
 * TB_ERR_NO_DEVICE.  On error *out is NULL and nothing is allocated. */
tb_status tb_create(tb_handle **out, const tb_system_desc *desc, void *stream);

/*
 * Ragged batch: n_systems independent systems (for example liquid-water
 * boxes of different sizes) in one handle.  They are placed block-diagonally
 * -- atoms and orbitals numbered system after system, no block couples two
 * systems -- so the Krylov space of a column e_j never leaves its system,
 * and every solve, Mulliken, CSC and Lanczos call takes columns of any
 * system of the batch in one launch sequence, with the results of separate
 * per-system solves (up to rounding order).  Every desc is validated as by
 * tb_create; H_vals must be given for all systems or for none, and with
 * none (Eq. Hap-1 on the device) all K must be equal.  Errors as tb_create.
 */
tb_status tb_create_batch(tb_handle **out, const tb_system_desc *descs, int32_t n_systems, void *stream);

/* Systems of a handle (1 for tb_create) and their first atom / orbital:
 * atom_off, orb_off: host int64 [n_systems + 1] (either may be NULL). */
int32_t tb_num_systems(const tb_handle *h);
tb_status tb_batch_offsets(const tb_handle *h, int64_t *atom_off, int64_t *orb_off);

/*
 * Bounds [lo, hi] of the spectrum of S used by the Chebyshev corrections of
 * TB_MIXED: extreme Ritz values of an 80-step Lanczos run on S (host, FP64,
 * computed once per handle), widened by their residual norms and by 3 % /
 * 1 %.  lo <= 0 means no usable lower bound (the FP32 CG corrections are
 * used).  TB_ERR_S_NOT_SPD if a Ritz value of S is <= 0.
 */
tb_status tb_overlap_bounds(tb_handle *h, double *lo, double *hi);

/*
 * The same bounds for a system description, on the host only (no device,
 * no handle): d as for tb_create (S_vals used, assumed symmetric; H_vals,
 * eps and K ignored).  TB_ERR_INVALID_ARG for a malformed pattern.
 */
tb_status tb_overlap_bounds_desc(const tb_system_desc *d, double *lo, double *hi);

/*
 * Chebyshev plan of the TB_MIXED corrections for spectrum bounds [lo, hi]
 * (host only): n (odd) steps per round reduce the error by at least
 * 1 / T_n(1 / sigma) <= lo_tol, sigma = (hi - lo) / (hi + lo); rounds =
 * ceil(log inner_tol / log lo_tol) rounds are planned, the last of n_last
 * <= n steps (enough for half the remaining reduction); gamma = 2 / (lo + hi);
 * omega[k] (1 <= k < n; omega[0] = 0) the step coefficients of the
 * recurrence d_{k+1} = d_{k-1} + omega[k] (gamma (f - S d_k) + d_k - d_{k-1}),
 * d_0 = 0, d_1 = gamma f.  omega: float [omega_len] or NULL.  *n = 0 when
 * lo <= 0, hi <= lo or n > cap (the FP32 CG corrections are used then).
 * A column that ends the planned rounds above inner_tol (the double-float
 * residual of the refinement is only good to ~2^-47 |S| |x|) runs up to two
 * more rounds of n_last steps, each checked by a residual with FP64
 * products, then FP32 CG rounds.
 */
tb_status tb_chebyshev_plan(double lo, double hi, double lo_tol, double inner_tol, int32_t cap, int32_t *n,
                            int32_t *n_last, int32_t *rounds, double *gamma, float *omega, int32_t omega_len);

/* Release all device memory of the handle (NULL is allowed). */
tb_status tb_destroy(tb_handle *h);

/* Number of orbitals N and atoms of the system. */
int64_t tb_num_orbitals(const tb_handle *h);
int64_t tb_num_atoms(const tb_handle *h);
int64_t tb_num_blocks(const tb_handle *h);

typedef struct {
    double tol;               /* shift converged when ||r_{n+1}||_2/|pi^k_{n+1}| <= tol
                                 (||e_j|| = 1); default 1e-10                         */
    double inner_tol;         /* inner CG: ||r - S r'|| <= inner_tol ||r||; 1e-13      */
    int32_t max_iter;         /* outer iterations per panel; default 100000           */
    int32_t inner_max_iter;   /* inner CG iterations per outer step; default 1000     */
    int32_t panel;            /* right-hand sides per panel (power of two <= 256);
                                 0 = automatic                                         */
    int32_t seed;             /* index of the initial seed shift; default 0           */
    int32_t switching;        /* 1 = seed switching (default), 0 = keep the seed       */
    int32_t force_switch_every; /* > 0: also switch every that many steps (testing)    */
    int32_t precision;        /* TB_FP64 (default): every product in FP64;
                                 TB_MIXED: the inner solve S r' = r runs as FP32
                                 corrections (inner_method) inside FP64 iterative refinement
                                 (residual r - S r' in FP64 each round) until
                                 ||r - S r'|| <= inner_tol ||r||; all other steps FP64 */
    double inner_lo_tol;      /* TB_MIXED: relative tolerance of each FP32 correction round;
                                 default 1e-6                                            */
    int32_t inner_method;     /* TB_MIXED: how the FP32 corrections of a round are made.
                                 TB_INNER_CHEBYSHEV (default): a fixed number of
                                 Chebyshev steps for the spectrum of S (bounds from a
                                 Lanczos run on S on the host, once per handle), enough
                                 to reduce the error by inner_lo_tol, each step one
                                 kernel with no inner products; from the fourth round on
                                 (and for an S whose bounds are unusable) FP32 CG.
                                 TB_INNER_CG: FP32 CG in every round.  Either way the
                                 FP64 residual of each round decides convergence, so both
                                 reach the same inner_tol.  Ignored for TB_FP64 (CG).   */
    int64_t state_bytes;      /* energy-point checkpointing: device bytes allowed for the
                                 full-vector state of the shifts (x^k and p^k of every
                                 shift for the columns in flight, plus the device copy of
                                 the full solutions; tb_shifted_cocg and tb_mulliken_vjp).
                                 When all K shifts would exceed it, the shifts are taken
                                 in chunks, each a separate shifted solve of the same
                                 columns whose seed sequence is recomputed (its seed is
                                 the chunk's own first shift, or opts->seed inside the
                                 chunk that holds it); each chunk's solutions go to the
                                 caller's output -- host memory included -- before the
                                 next chunk starts, so state_bytes bounds device memory
                                 whatever K.  Every shift's solution is the same to tol
                                 as in one call.  0 = 8 GiB (default).                    */
} tb_solve_opts;

/* Fill *opts with the defaults listed above. */
enum { TB_INNER_CHEBYSHEV = 0, TB_INNER_CG = 1 };

void tb_default_opts(tb_solve_opts *opts);

/* Optional statistics; every pointer member may be NULL. */
typedef struct {
    int32_t *conv_iter;        /* host [R*K]: outer step at which shift k of column
                                  c converged (index c*K + k), -1 if it did not      */
    int64_t outer_iterations;  /* sum over columns of the steps each column ran    */
    int64_t inner_iterations;  /* sum over outer steps of inner CG iterations       */
    int64_t max_column_iterations; /* steps of the slowest column                   */
    int32_t switches;          /* seed switches, all columns                       */
    int32_t unconverged;       /* (column, shift) pairs not converged              */
    double seconds;            /* wall time of the solve                           */
    int32_t inner_redos;       /* TB_MIXED: inner solves whose FP32 corrections did
                                  not converge and were redone with the FP64 CG     */
} tb_stats;

/*
 * Full solutions.  For shifts z[0..K-1] (host, complex) and right-hand sides
 * e_j, j = cols[0..R-1] (host), writes
 *     x_out[(k*R + c)*N + i] = (x_{cols[c]}(z_k))_i     (complex, host or device)
 * Memory for x_out: K*R*N complex doubles.
 * Returns TB_ERR_NOT_CONVERGED if some shift did not reach opts->tol within
 * max_iter steps (the converged ones are valid), TB_ERR_BREAKDOWN or
 * TB_ERR_S_NOT_SPD if the iteration failed.
 */
tb_status tb_shifted_cocg(tb_handle *h, int32_t K, const double *z, int32_t R, const int32_t *cols,
                          const tb_solve_opts *opts, double *x_out, tb_stats *stats, void *stream);

/*
 * Launch autotuner (no counterpart in the paper: a choice of how the work of
 * a call is laid out on the GPU, not of what it computes).  For this
 * handle's system and the shift set z (K shifts) it times, for
 * `iters` outer iterations of Mulliken-projected solves with weights w
 * (tb_mulliken_orbital's work), every candidate of
 *   panel width P in {32, 64, 128, 256} (not above the orbital count),
 *   panels in flight (worker streams) in {2, 4}, and, on the mixed path
 *   with Chebyshev corrections, the Chebyshev-step form: 4 complex columns
 *   per thread at 3 resident CTAs per SM, or 2 at 4 CTAs per SM,
 * on P x (panels in flight) columns spread evenly over the system (an
 * untimed call first builds the graphs and the spectrum bounds; CUDA events
 * on `stream` time the second).  The best choice is kept in the handle for
 * the size class (opts->precision, opts->inner_method, K rounded up to a
 * power of two): later calls with opts->panel == 0 use its panel width,
 * panels in flight and step form.  out[0 .. *n_out) receives the candidates
 * ordered by rate, best first (at most max_out).  Other fields of opts
 * (tolerances, precision) apply to the trial solves; max_iter is replaced by
 * iters.  Status as tb_mulliken_orbital (not converging within iters is
 * expected and not an error).
 */
typedef struct {
    int32_t panel;        /* right-hand sides per panel                          */
    int32_t streams;      /* panels in flight                                    */
    int32_t cheb_cpt;     /* complex columns per thread of the Chebyshev step (0: not used) */
    int32_t ctas_per_sm;  /* resident CTAs per SM of that step (0: not used)     */
    double rate;          /* measured shift*RHS*iterations per second            */
} tb_tune;
tb_status tb_autotune(tb_handle *h, int32_t K, const double *z, const double *w, double g_s,
                      const tb_solve_opts *opts, int32_t iters, tb_tune *out, int32_t max_out, int32_t *n_out,
                      void *stream);

/*
 * Selected Green's-function elements (Eq. GreensFunc) with the shifted
 * solutions projected on the requested rows (no full solution is stored).
 * Column c (orbital cols[c]) asks for rows rows[row_ptr[c] .. row_ptr[c+1]-1]
 * (host arrays; row_ptr[0] = 0).  Writes, complex, host or device,
 *     G_out[(row_ptr[c] + r)*K + k] = G_{rows[row_ptr[c]+r], cols[c]}(z_k).
 * At most 1024 rows per column.  Status as tb_shifted_cocg.
 */
tb_status tb_green_elements(tb_handle *h, int32_t K, const double *z, int32_t R, const int32_t *cols,
                            const int64_t *row_ptr, const int32_t *rows, const tb_solve_opts *opts,
                            double *G_out, tb_stats *stats, void *stream);

/*
 * As tb_green_elements, and also dG_ij/dz at the same elements (the
 * adjoint building block; dG/dz = -G S G).  The derivative is carried
 * through the same Krylov sequence by differentiating the shift recurrences
 * (Eq. shift:pi and the alpha^k, beta^k relations) with respect to z_k with
 * the seed quantities fixed: no extra matrix products, 2x the per-shift
 * state.  dG_out: complex [row_ptr[R]][K] like G_out, host or device.
 */
tb_status tb_green_elements_dz(tb_handle *h, int32_t K, const double *z, int32_t R, const int32_t *cols,
                               const int64_t *row_ptr, const int32_t *rows, const tb_solve_opts *opts,
                               double *G_out, double *dG_out, tb_stats *stats, void *stream);

/*
 * Band-structure energy and its gradients (adjoint; the quadrature z_k,
 * w_k must have real weights):
 *     E = Tr(rho H) = -(g_s/pi) Im sum_k w_k z_k Tr[G(z_k) S],
 *     dE/dH_ab = -(g_s/pi) Im sum_k w_k z_k [G S G]_ba,
 *     dE/dS_ab = -(g_s/pi) Im sum_k w_k (z_k G_ba - z_k^2 [G S G]_ba),
 * H_ab, S_ab taken as independent entries of the stored pattern.  All N
 * columns are solved with their pattern rows projected (values and z-
 * derivatives, as tb_green_elements_dz).  E_out: one double; dE_dH, dE_dS:
 * double arrays in the caller's block layout of S_vals (one value per
 * stored entry); host or device.  Chain rule to forces (dS/dR, dH/dR) is the
 * caller's.  Status as tb_shifted_cocg; TB_ERR_INVALID_ARG if a block
 * column holds more than 1024 orbitals.
 */
tb_status tb_band_energy(tb_handle *h, int32_t K, const double *z, const double *w, double g_s,
                         const tb_solve_opts *opts, double *E_out, double *dE_dH, double *dE_dS, tb_stats *stats,
                         void *stream);

/*
 * Forces F_I = -dE/dR_I from the band-energy gradients of tb_band_energy
 * (chain rule through the geometry): every stored entry e of an off-site
 * block (I, J) contributes v_e = dE/dS_e dS_e/dd + dE/dH_e dH_e/dd, with
 * d = R_J - R_I the block's bond vector, as F_I += v_e, F_J -= v_e; on-site
 * blocks do not move.  dE_dH, dE_dS: double [n_values] (tb_band_energy's
 * outputs); dS_dd, dH_dd: double [3][n_values], the caller's geometry
 * derivatives of every stored entry (component-major); dH_dd == NULL uses
 * Eq. Hap-1, dH_e/dd = K (eps_a + eps_b)/2 dS_e/dd (handles whose H was
 * built from eps and K only, else TB_ERR_INVALID_ARG).  The charge-transfer
 * term of Eq. Hap-CSC is not included.  F_out: double [n_atoms][3]; all
 * arrays host or device.
 */
tb_status tb_forces(tb_handle *h, const double *dE_dH, const double *dE_dS, const double *dS_dd,
                    const double *dH_dd, double *F_out, void *stream);

/*
 * Vector-Jacobian product of the Mulliken populations (adjoint): for
 * L = sum_a v_a q_a, q_a the gross population of orbital a (v: double [N]
 * weights, host or device; per-atom charges take v_a = the atom's weight on
 * each of its orbitals),
 *     dL/dH_ab = -(g_s/pi) Im sum_k w_k [G S D_v G]_ba,
 *     dL/dS_ab = -(g_s/pi) Im sum_k w_k (v_b G_ba - z_k [G S D_v G]_ba),
 * D_v = diag(v), at every stored entry (the caller's block layout).  It needs
 * full-vector shifted solves with right-hand sides e_c and s_c (column c of
 * S) for every orbital c with v_c != 0, contracted on the pattern:
 * [G S D_v G]_ba = sum_c v_c (G s_c)_b (G e_c)_a -- 2 m full-vector solves
 * and O(m K nnz) work for m nonzero weights: cheap for a local L (a few
 * atoms' charges) on any system size, O(N K nnz) for weights on every
 * orbital.  Solves use opts; status as
 * tb_shifted_cocg; a batch handle of more than one system is
 * TB_ERR_INVALID_ARG.  dL_dH, dL_dS: double [n_values], host or device.
 */
tb_status tb_mulliken_vjp(tb_handle *h, int32_t K, const double *z, const double *w, double g_s, const double *v,
                          const tb_solve_opts *opts, double *dL_dH, double *dL_dS, tb_stats *stats, void *stream);

/*
 * Gross Mulliken populations of selected orbitals (Section 2.2, the
 * Mulliken partition of the charge density), from the energy integral of
 * the Green's function with the quadrature (z_k, w_k) (host, complex):
 *     q_j = -(g_s/pi) Im sum_k w_k (G(z_k) S)_jj = -(g_s/pi) Im sum_k w_k s_j^T x_j(z_k),
 * s_j the j-th column of S.  Writes q_out[c] for orbital cols[c]
 * (double, host or device).  Status as tb_shifted_cocg.
 */
tb_status tb_mulliken_orbital(tb_handle *h, int32_t K, const double *z, const double *w, double g_s,
                              int32_t R, const int32_t *cols, const tb_solve_opts *opts,
                              double *q_out, tb_stats *stats, void *stream);

/*
 * Gross Mulliken population of every atom: q_i = sum of q_j over the
 * orbitals j of atom i, all N orbitals solved in panels.  q_out: double
 * [n_atoms], host or device.  Status as tb_shifted_cocg.
 */
tb_status tb_mulliken_charges(tb_handle *h, int32_t K, const double *z, const double *w, double g_s,
                              const tb_solve_opts *opts, double *q_out, tb_stats *stats, void *stream);

/* ---- charge self-consistency (Section 2.2, Eq. Hap-CSC) ------------------
 *
 * The charge-transfer term of the Hamiltonian,
 *     H^CSC_{ia,jb} = 1/2 S_{ia,jb} sum_k (gamma_ik + gamma_jk) dq_k
 *                   = 1/2 S_{ia,jb} (V_i + V_j),   V = gamma dq,
 * with dq_k the deviation of the Mulliken population of atom k from a
 * reference and gamma the atom-atom Coulomb interaction (chemical hardness
 * on the diagonal).  The paper fixes neither gamma nor the iteration that
 * makes the charges self-consistent: gamma is the caller's dense matrix and
 * the iteration is linear mixing of dq.  The handle keeps the Hamiltonian
 * it was created with (H0: explicit or ASED, Eq. Hap-1); these calls
 * replace the Hamiltonian that every solve uses by H0 + H^CSC(dq).
 */
typedef struct {
    int32_t max_scf;   /* SCF iterations, >= 1; default 50                          */
    double scf_tol;    /* stop when max_i |dq_out_i - dq_in_i| <= scf_tol (electrons),
                          > 0; default 1e-6                                         */
    double mix;        /* dq_in <- dq_in + mix (dq_out - dq_in), 0 < mix <= 1;
                          default 0.3                                               */
} tb_csc_opts;

/* Fill *opts with the defaults listed above. */
void tb_default_csc_opts(tb_csc_opts *opts);

typedef struct {
    int32_t iterations;        /* SCF iterations run                                */
    double residual;           /* max_i |dq_out_i - dq_in_i| of the last iteration  */
    int64_t outer_iterations;  /* COCG outer steps summed over all SCF iterations   */
    int64_t inner_iterations;  /* inner CG iterations summed likewise               */
    double seconds;            /* wall time of the loop                             */
} tb_csc_stats;

/*
 * Set the handle's Hamiltonian to H0 + H^CSC(dq): V = gamma dq on the device,
 * then every stored block H_IJ = H0_IJ + 1/2 S_IJ (V_I + V_J) (and its FP32
 * split for TB_MIXED).  gamma: double [n_atoms][n_atoms] row-major; dq:
 * double [n_atoms]; either may be host or device memory.  dq == NULL
 * restores H0 (gamma is then ignored).  Synchronous on the stream.
 */
tb_status tb_csc_hamiltonian(tb_handle *h, const double *gamma, const double *dq, void *stream);

/*
 * Self-consistent Mulliken charges by linear mixing.  Iteration m sets
 * H = H0 + H^CSC(dq_in) (dq_in = dq_init, or 0 when dq_init is NULL, at
 * m = 1), computes the atomic populations q as tb_mulliken_charges does
 * (quadrature z, w; spin factor g_s; solver options opts), dq_out = q - q_ref
 * and res = max_i |dq_out_i - dq_in_i|; it stops when res <= scf_tol or
 * m = max_scf, else dq_in <- dq_in + mix (dq_out - dq_in).  Every step runs
 * on the device; the host reads one number (res) per iteration.
 * Inputs gamma [n_atoms][n_atoms], q_ref [n_atoms], dq_init [n_atoms]
 * (optional): host or device.  Outputs q_out, dq_out [n_atoms], host or
 * device: the populations of the last iteration and the dq_in that produced
 * them; on return the handle's Hamiltonian is H0 + H^CSC(dq_out).
 * Returns TB_OK when res <= scf_tol, TB_ERR_NOT_CONVERGED when max_scf ran
 * out or a COCG solve did not converge (outputs still written),
 * TB_ERR_BREAKDOWN on a non-finite residual, TB_ERR_INVALID_ARG for bad
 * options, and the errors of tb_mulliken_charges.
 */
tb_status tb_csc_loop(tb_handle *h, int32_t K, const double *z, const double *w, double g_s,
                      const double *gamma, const double *q_ref, const double *dq_init,
                      const tb_csc_opts *copts, const tb_solve_opts *opts, double *q_out, double *dq_out,
                      tb_csc_stats *stats, void *stream);

/*
 * Forces of the charge-self-consistent model (Section 2.2, Eq. Hap-CSC; the
 * paper cites the second-order charge-transfer energy but prints no total
 * energy).  With the quadrature (z_k, w_k) the occupation is smeared, and
 * the functional whose H-derivative is exactly the density matrix is the
 * contour grand potential Omega(H, S) = (g_s/pi) Im sum_k w_k Tr ln(z_k S - H);
 * the free energy A(dq) = Omega(H0 + H^CSC(dq), S) - V^T (dq + q_ref)
 * + 1/2 dq^T gamma dq (V = gamma dq) has dA/d dq = gamma (q_out - q_in), so at
 * a self-consistent dq (tb_csc_loop's dq_out) the forces need no charge
 * response:
 *     F_I = -dA/dR_I = -sum_ab [rho_ba dH0_ab/dR_I + (dOmega/dS_ab
 *           + rho_ba (V_a + V_b)/2) dS_ab/dR_I] - dq_I sum_k (dgamma_Ik/dR_I) dq_k,
 * rho = -(g_s/pi) Im sum_k w_k G(z_k), dOmega/dS_ab = (g_s/pi) Im sum_k
 * w_k z_k G_ba(z_k), H0 by Eq. Hap-1 (handles built from eps and K only, else
 * TB_ERR_INVALID_ARG).  The call sets the handle's H to H0 + H^CSC(dq) (as
 * tb_csc_hamiltonian, and leaves it there), solves every column with the
 * rows of its block column projected, and applies the force kernels of
 * tb_forces plus the Coulomb-gradient term.  gamma: double [n_atoms][n_atoms];
 * dgamma: double [n_atoms][n_atoms][3], d gamma_Ik / d R_I; dq: double
 * [n_atoms]; dS_dd: double [3][n_values] as in tb_forces; F_out: double
 * [n_atoms][3]; all host or device.  Status as tb_shifted_cocg; a batch
 * handle of more than one system is TB_ERR_INVALID_ARG.
 */
tb_status tb_csc_forces(tb_handle *h, int32_t K, const double *z, const double *w, double g_s,
                        const double *gamma, const double *dgamma, const double *dq, const double *dS_dd,
                        const tb_solve_opts *opts, double *F_out, tb_stats *stats, void *stream);

/*
 * Generalized Lanczos process (Section 3.2, Eqs. 1.13 and 1.18) for the
 * operator S^-1 H with the S-product, started from u^0 = S^-1 e_j normalised
 * in the S-norm.  Writes a[0..n_steps-1], b[0..n_steps] (b[0] = 0) and
 * *norm = e_j^T S^-1 e_j (all double, host or device), so that
 *     G_jj(z) = norm / (z - a_0 - b_1^2 / (z - a_1 - b_2^2 / ...)).
 * If some b_{n+1} is 0 the remaining coefficients are 0 (invariant
 * subspace found).  inner_tol as in tb_solve_opts (<= 0: 1e-13).
 */
tb_status tb_generalized_lanczos(tb_handle *h, int32_t j, int32_t n_steps, double inner_tol,
                                 double *a, double *b, double *norm, void *stream);

/*
 * Diagonal Green's function element from Lanczos coefficients (Section 3.2:
 * G in the generalized Krylov subspace), the continued fraction
 *     G_jj(z_k) = norm / (z_k - a_0 - b_1^2 / (z_k - a_1 - ... - b_{n-1}^2 / (z_k - a_{n-1})))
 * evaluated bottom-up on the device for K points; the local density of
 * states is -Im G_jj(E + i eta) / pi.  a [n_steps], b [n_steps + 1] as
 * written by tb_generalized_lanczos (host or device); z: host, complex
 * (interleaved re, im) [K]; G_out: complex [K], host or device.
 */
tb_status tb_lanczos_green(const double *a, const double *b, double norm, int32_t n_steps, int32_t K,
                           const double *z, double *G_out, void *stream);

/*
 * Generalized Lanczos for R columns at once: R independent processes (one
 * per e_{cols[c]}) run together on panels of opts->panel columns (0: 64),
 * their S^-1 products solved as one panel (opts->precision selects the FP64
 * CG or FP32 CG inside FP64 refinement; opts->inner_tol their accuracy).
 * Writes a[c][0..n_steps-1], b[c][0..n_steps] (b[c][0] = 0) and norm[c], in
 * the layout and meaning of tb_generalized_lanczos (host or device).
 * tb_generalized_lanczos(h, j, ...) is the case R = 1 in FP64.
 */
tb_status tb_generalized_lanczos_batch(tb_handle *h, int32_t R, const int32_t *cols, int32_t n_steps,
                                       const tb_solve_opts *opts, double *a, double *b, double *norm,
                                       void *stream);

/*
 * tb_lanczos_green for R processes at once (the outputs of
 * tb_generalized_lanczos_batch): a [R][n_steps], b [R][n_steps + 1],
 * norm [R] (host or device), z host complex [K]; G_out complex [R][K].
 */
tb_status tb_lanczos_green_batch(int32_t R, const double *a, const double *b, const double *norm, int32_t n_steps,
                                 int32_t K, const double *z, double *G_out, void *stream);

/*
 * Allocation-free generalized Lanczos.  The paper has no counterpart: this
 * entry point exists for callers that cannot allocate GPU memory while they
 * call the library -- for example code that runs with the whole device
 * memory already handed to another allocator, or that must not touch the
 * allocator at all (a real-time loop that may not block on cudaMalloc, or a
 * host that only hands over buffers it owns).  It takes the same arguments
 * and gives the same results and errors as tb_generalized_lanczos, but it
 * calls no cudaMalloc, cudaFree or other allocating routine: its scratch
 * memory is one fixed device array inside the library,
 * TB_NOALLOC_SCRATCH_BYTES (16 MiB) long.  The handle (made by tb_create,
 * which does allocate) and the outputs a, b, norm are the caller's.
 *  - Set-up: tb_create places the array on the handle's device, looks up its
 *    device address (cudaGetSymbolAddress, with that device current) and
 *    loads the kernels this call launches (with CUDA's lazy module loading
 *    both would otherwise happen, and allocate, at the first call).  Every
 *    GPU on which a handle was created holds the array until the process
 *    exits.  Call this entry point with the handle's device current
 *    (otherwise TB_ERR_INVALID_ARG).
 *  - Size limit: the call needs about 160 * 4 * n_atoms + 16 * n_steps bytes
 *    (plus ~50 kB); a request that does not fit returns TB_ERR_TOO_LARGE
 *    before any device work (N up to ~100 000 orbitals with a few hundred
 *    steps).
 *  - All calls share the one array and it keeps the previous call's
 *    contents (each call clears what it needs zeroed).  Calls whose GPU work
 *    overlaps -- on different streams or from different threads, with this
 *    or any other handle -- race on it; serialise them.
 *  - Kernel timing (tb_profile_enable(1)) creates CUDA events on first use;
 *    leave it off in callers that must not allocate.
 */
#define TB_NOALLOC_SCRATCH_BYTES (16u << 20)
tb_status tb_generalized_lanczos_noalloc(tb_handle *h, int32_t j, int32_t n_steps, double inner_tol,
                                         double *a, double *b, double *norm, void *stream);

/*
 * Launch accounting for measurement tools (no counterpart in the paper).
 * tb_launch_count: number of kernels this library has launched since it was
 * loaded (all threads, all devices).
 * tb_profile_enable(1) resets the per-kernel totals and from then on
 * brackets every launch with a pair of CUDA events on the launch's stream;
 * tb_profile_enable(0) stops it.  tb_profile_read waits for the recorded
 * events and returns, for one kernel class TB_K_*, the launches counted since
 * the last reset and their summed device time in milliseconds (0 ms while
 * profiling is off).  Counting is thread-safe (the library's own worker
 * threads launch concurrently); enable, read and reset from one thread.
 */
enum {
    TB_K_INNER_SPMV = 0,   /* w = S r and the inner-CG dot products        */
    TB_K_INNER_UPDATE = 1, /* inner-CG vector updates                      */
    TB_K_OUTER_SPMM = 2,   /* q = (z_s S - H) r', A p and mu               */
    TB_K_OUTER_UPDATE = 3, /* r_{n+1} = r_n - alpha A p                    */
    TB_K_FINISH = 4,       /* rho_{n+1}                                    */
    TB_K_SHIFT_STEP = 5,   /* all shifts, projections, seed switching      */
    TB_K_FULL_UPDATE = 6,  /* full-mode x^k, p^k updates                   */
    TB_K_OTHER = 7,        /* set-up, outputs, Lanczos helpers             */
    TB_K_INNER32_SPMV = 8, /* TB_MIXED: FP32 w = S r and dot products      */
    TB_K_INNER32_UPDATE = 9, /* TB_MIXED: FP32 CG vector updates (and the
                              first Chebyshev step)                           */
    TB_K_REFINE_RESIDUAL = 10, /* TB_MIXED: FP64 residual r - S r'         */
    TB_K_REFINE_AUX = 11,  /* TB_MIXED: refinement start and correction add */
    TB_K_CSC = 12,         /* charge self-consistency: potential, Hamiltonian
                              update, atom sums, mixing                        */
    TB_K_INNER32_CHEB = 13, /* TB_MIXED: one Chebyshev correction step (FP32
                              S d and the update of d in one kernel)          */
    TB_K_COUNT = 14
};
/*
 * FMA throughput of the current device, measured (no counterpart in the
 * paper: the denominator of the roofline fractions of ALU-bound kernels).
 * mode 0: scalar FP32 FMA, 1: packed FP32 FMA (two lanes per instruction),
 * 2: FP64 FMA; 8 independent register chains per thread, 64 warps per SM,
 * one timed launch after a warm-up (CUDA events on `stream`).  Writes
 * TFLOP/s (2 flop per multiply-add) to *tflops_out.
 */
tb_status tb_measure_fma_peak(int32_t mode, double *tflops_out, void *stream);

int64_t tb_launch_count(void);
void tb_profile_enable(int32_t enable);
tb_status tb_profile_read(int32_t kernel, int64_t *launches, double *total_ms);
/* Busy time (ms) of a kernel class since profiling was enabled: the union
 * of its launch intervals, so overlapping launches on several streams (two
 * panels in flight, ragged batches) count once.  0 without profiling. */
tb_status tb_profile_busy(int32_t kernel, double *busy_ms);

/* Static string naming a status code. */
const char *tb_status_string(tb_status s);

#ifdef __cplusplus
}
#endif

#endif /* TBCOCG_H */
