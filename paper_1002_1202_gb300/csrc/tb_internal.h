// Internal declarations shared by the kernels (tb_kernels.cu) and the host
// orchestration (tb_api.cu).  Nothing here is part of the public C ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

namespace tb {

constexpr int THREADS = 256;   // every kernel runs 256-thread CTAs
constexpr int MAX_P = 256;     // right-hand sides per panel (power of two)
constexpr int MAX_K = 1024;    // shifts per call
constexpr int MAX_M = 1024;    // projected rows per column

constexpr int NFLAGS = 8;      // device status words of a panel (see PanelDev::flags)
constexpr int NPOOL = 8;       // host worker threads of one call, at most
constexpr int RED_GROUP = 32;  // CTAs per first-level group of the grid reductions
constexpr int MAX_GROUPS = 64; // upper bound on first-level groups (grids <= 2048 CTAs)
constexpr int HIST_IT = 64;    // FP32 CG iterations kept by the trace history

// error bits in PanelDev::flags[0]
constexpr int ERR_BREAKDOWN = 1;   // COCG breakdown of the outer recurrence (mu or rho zero / non-finite)
constexpr int ERR_NOT_SPD = 2;
constexpr int ERR_INNER = 4;       // mixed path: a refinement residual of the inner solve went non-finite

// functional kinds of the projected mode
constexpr int PROJ_NONE = 0;   // full solutions kept (x^k, p^k are N-vectors)
constexpr int PROJ_ROWS = 1;   // G elements: unit vectors e_row
constexpr int PROJ_SROW = 2;   // Mulliken: s_j = row j of S (one functional)

// Device copy of the block-sparse system.  Atoms are padded to 4 orbital
// slots (s, px, py, pz); a padded slot has S = 1 on its diagonal and no
// coupling, so it stays exactly zero in every vector.
struct DevSystem {
    int n_atoms = 0;
    int64_t nb = 0;
    int npad = 0;              // 4 * n_atoms
    int* brow = nullptr;       // [n_atoms + 1]
    int* bcol = nullptr;       // [nb]
    double* S = nullptr;       // [nb][16] row-major 4x4 blocks
    double* H = nullptr;       // [nb][16]
    float* S32 = nullptr;      // [nb][16] S rounded to FP32 (S_hi of the double-float split)
    float* S32lo = nullptr;    // [nb][16] S - S_hi in FP32
    float* S32T = nullptr;     // [nb][16] S_hi of every block transposed (column e of the block as row e)
    // Exact orbital counts for the Chebyshev step of systems with s-only
    // atoms (rag = 1; absent for all-sp systems): the orbital count of every
    // atom, the block rows in the order sp atoms first, then s atoms (one
    // run of each kind per system, so a warp's rows are of one kind), and
    // the FP32 blocks stored with their real entries only, at 16-byte
    // aligned float offsets: 4x4 transposed (column e as row e), 4x1 as the
    // column S[0..3][0], 1x4 as the row S[0][0..3], 1x1 as S[0][0] and three
    // zeros.
    int rag = 0;
    // 1 when every block row holds its diagonal block once, that block of S
    // is exactly the identity (orthonormal orbitals on one atom, as an STO
    // basis gives) and no atom has a single orbital: the FP32 Chebyshev
    // steps then skip the diagonal block and add the vector's own rows.
    int unit_diag = 0;
    unsigned char* norb = nullptr;   // [n_atoms] 1 or 4
    int* row_order = nullptr;        // [n_atoms] atom of each block-row slot (indices of this view)
    float* S32r = nullptr;           // compact blocks
    int2* bmeta = nullptr;           // [nb] per block: x = block-column atom (index of this view),
                                     // y = offset of the block in S32r in float4 units, bit 31 set
                                     // when the column atom has one orbital
    float* H32hi = nullptr;    // [nb][16] H rounded to FP32
    float* H32lo = nullptr;    // [nb][16] H - H_hi in FP32
    // atom groups of the grouped FP32 SpMV: group g = atoms [g * grpG, (g + 1) * grpG)
    int grpG = 0;              // atoms per group; 0: grouped SpMV not used
    int n_groups = 0;
    int max_union = 0;         // largest number of distinct block columns of a group
    int max_gblocks = 0;       // largest number of blocks of a group
    int* grp_ptr = nullptr;    // [n_groups + 1] offsets into grp_cols
    int* grp_cols = nullptr;   // distinct block-column atoms of each group, ascending
    int* blk_loc = nullptr;    // [nb] position of bcol[b] in the list of its group
};
size_t inner32_grp_smem(const DevSystem& s);   // dynamic shared memory of the grouped SpMV

// Per right-hand side (complex column) state of a panel.
struct ColState {
    double2 zs;          // seed shift z_s
    double2 alpha;       // alpha_n of the current step
    double2 alpha_prev;  // alpha_{n-1}
    double2 beta_prev;   // beta_{n-1}
    double2 rho;         // rho_n = r_n^T r'_n
    double2 rho_new;     // rho_{n+1}
    double2 sc_cur;      // pending scale of r_n and r'_n (seed switch)
    double2 sc_prev;     // pending scale of r_{n-1}
    double rnorm;        // ||r_{n+1}||_2
    int32_t seed;        // index of the seed shift
    int32_t active;      // 1 while some shift of the column is unconverged
    int32_t iters;       // outer steps run
    int32_t switches;    // seed switches
    int32_t row;         // padded orbital index of e_j, -1 for a dummy column
    int32_t n_unconv;    // unconverged shifts
    int32_t nfun;        // projected functionals of this column
    int32_t pad_;
};

// Per real column (two per complex column) state of the inner CG.
struct InnerState {
    double gamma_prev;
    double alpha;
    double beta;
    double bnorm2;
    int32_t conv;
    int32_t skip;        // refinement: this real column needs no further correction
    double scale;        // refinement: FP32 right-hand side = FP64 residual * scale
    double unscale;      // refinement: 1 / scale (the residual norm; 0 when skipped), the
                         // factor of the correction, so no kernel divides per element
};

struct PanelDev {
    int P = 0, K = 0, npad = 0, M = 0, proj = PROJ_NONE;
    int grid = 0;                 // CTAs of the grid-stride kernels
    int mixed = 0;                // 1: inner S^-1 by FP32 corrections inside FP64 refinement
    int cheb_cpt = 0;             // host side: columns per thread of the Chebyshev step (2 or 4; 0 = default)
    double tol = 1e-10, inner_tol = 1e-13, inner_lo_tol = 1e-6;
    int switching = 1, force_switch_every = 0;
    // panel vectors, [npad][P] complex
    double2 *Rcur = nullptr, *Rprev = nullptr, *Rp = nullptr, *W = nullptr;
    double2 *Rin = nullptr, *Pin = nullptr, *Sin = nullptr;
    float4* RpS = nullptr;        // mixed: r' split (re_hi, re_lo, im_hi, im_lo) for double-float SpMVs
    // FP32 inner CG of the mixed-precision solve, [npad][P] complex floats
    float2 *r32 = nullptr, *p32 = nullptr, *s32 = nullptr, *w32 = nullptr, *x32 = nullptr;
    InnerState* inner32 = nullptr; // [3][2P]: refinement state, CG state slots 0 and 1
    double* acc32 = nullptr;       // [2][4][P]: FP32 CG sums (gamma, delta per real column), two slots
    double* cgs = nullptr;         // [2][2P]: alpha, beta of the current FP32 CG iteration
    unsigned char* cgu = nullptr;  // [2P]: real column updated in the current FP32 CG iteration
    unsigned* ticket32 = nullptr;  // [1]: completion ticket of the FP32 SpMV (0 between launches)
    ColState* col = nullptr;       // [P]
    InnerState* inner = nullptr;   // [2P]
    double2* z = nullptr;          // [K]
    double2 *pi = nullptr, *pi_prev = nullptr;   // [P][K]
    int32_t* conv_iter = nullptr;                // [P][K]
    double2 *ak = nullptr, *bk = nullptr, *ipi = nullptr;  // [P][K] this step (full mode)
    int32_t* frow = nullptr;       // [P][M] padded rows (PROJ_ROWS)
    double2 *t = nullptr, *u = nullptr;          // [P][K][M] projected x, p
    int deriv = 0;                               // 1: also d/dz_k of the projections (PROJ_ROWS)
    double2 *dpi = nullptr, *dpi_prev = nullptr; // [P][K] d pi^k / d z_k
    double2 *dt = nullptr, *du = nullptr;        // [P][K][M] d/dz_k of t, u
    double2 *X = nullptr, *Pk = nullptr;         // [K][npad][P] full mode x, p
    double* partials = nullptr;    // [grid][4][P] per-CTA sums
    double* partials2 = nullptr;   // [MAX_GROUPS][4][P] per-group sums
    unsigned* counter = nullptr;   // [1 + MAX_GROUPS] arrival tickets of the grid reductions
    double* dbg = nullptr;         // [8] record of the first inner-CG breakdown (diagnostics)
    double* hist = nullptr;        // trace only: [HIST_IT][2P][4] gamma, delta, alpha, beta per FP32 CG iteration
    int* flags = nullptr;          // [NFLAGS]: 0 errors, 1 inner active, 2 active columns,
                                   // 3 inner iterations used, 4 refinement: unconverged real columns,
                                   // 5 FP32 CG rounds stopped early by a rounding breakdown,
                                   // 6 mixed inner solves redone with the FP64 CG,
                                   // 7 FP32 CG iteration whose scalars are current
};

// kernel classes for launch accounting (same order as the TB_K_* constants
// of the public header)
enum { K_INNER_SPMV = 0, K_INNER_UPDATE, K_OUTER_SPMM, K_OUTER_UPDATE, K_FINISH, K_SHIFT_STEP,
       K_FULL_UPDATE, K_OTHER, K_INNER32_SPMV, K_INNER32_UPDATE, K_REFINE_RESIDUAL, K_REFINE_AUX, K_CSC, K_INNER32_CHEB,
       K_COUNT };
void profile_enable(bool on);
void prof_harvest();
// launch accounting of a captured graph: the event pairs recorded by its
// nodes (one per captured launch) and the kernels each launch runs
struct GraphProf {
    std::vector<size_t> pairs;          // timed launches (profiling on at capture)
    std::vector<int> counts;
    std::vector<int> untimed_kid;       // launches captured with profiling off
    std::vector<int> untimed_counts;
};
void graph_prof_begin(GraphProf* gp);   // this thread's next captured launches get pairs in gp
void graph_prof_end();
void graph_prof_launched(const GraphProf& gp);
void graph_prof_release(GraphProf& gp);
void profile_read(int id, int64_t* launches, double* ms);
double profile_busy(int id);
int64_t launch_count();

// ---- launchers (tb_kernels.cu) -------------------------------------------
bool preload_noalloc_kernels();   // loads the allocation-free call's kernels onto the current device
void launch_ased_build(const DevSystem& s, const double* eps_pad, double K, cudaStream_t st);
void launch_split_f64(const double* v, float* hi, float* lo, long long n, cudaStream_t st);
void launch_transpose_blocks(const float* in, float* out, long long nb, cudaStream_t st);
void launch_compact_blocks(const DevSystem& s, cudaStream_t st);   // S32 -> S32r (rag systems)
void launch_panel_init(const DevSystem& s, const PanelDev& p, cudaStream_t st);
void launch_panel_rhs(const PanelDev& p, const double* rhs, const int32_t* orb2pad, int n_orb, int ncols,
                      cudaStream_t st);
void launch_vjp_accumulate(const double2* X, const double2* Y, int K, int Rc, int64_t N, const int32_t* cpos,
                           const double* vc, const int32_t* ea, const int32_t* eb, int64_t ne,
                           const double2* z, const double2* w, double g_s, double* gH, double* gS, cudaStream_t st);
// sx_from_residual (mixed path): Rin holds r_n - S r'_n from the refinement
void launch_outer_spmm(const DevSystem& s, const PanelDev& p, bool sx_from_residual, cudaStream_t st);
void launch_outer_update(const DevSystem& s, const PanelDev& p, cudaStream_t st);
void launch_inner_spmv(const DevSystem& s, const PanelDev& p, int it, cudaStream_t st);
void launch_inner_update(const DevSystem& s, const PanelDev& p, int it, cudaStream_t st);
void launch_finish(const DevSystem& s, const PanelDev& p, cudaStream_t st);
void launch_refine_start(const DevSystem& s, const PanelDev& p, const double2* b, cudaStream_t st);
// fp64: the residual with FP64 products (below the ~2^-47 relative floor of
// the double-float form) for the columns still above inner_tol
void launch_refine_residual(const DevSystem& s, const PanelDev& p, const double2* b, cudaStream_t st,
                            bool fp64 = false);
void launch_refine_add(const DevSystem& s, const PanelDev& p, cudaStream_t st);
void launch_refine_scale(const DevSystem& s, const PanelDev& p, const double2* src, float cheb_gamma, cudaStream_t st);
void launch_split_panel(const PanelDev& p, cudaStream_t st);
void launch_inner32_spmv(const DevSystem& s, const PanelDev& p, int it, cudaStream_t st);
void launch_inner32_cheb(const DevSystem& s, const PanelDev& p, const float2* cur, float2* io, float omega,
                         float gamma, int mode, cudaStream_t st);
// steps 1 .. n-1 of a Chebyshev round captured as a graph (false: not built)
bool cheb_graph_build(const DevSystem& s, const PanelDev& p, const float* omega, int n, float gamma,
                      cudaGraphExec_t* out);
void cheb_graph_launch(cudaGraphExec_t g, int steps, cudaStream_t st);
void cheb_graph_destroy(cudaGraphExec_t g);
void launch_inner32_update(const DevSystem& s, const PanelDev& p, int it, cudaStream_t st);
void launch_shift_init(const DevSystem& s, const PanelDev& p, cudaStream_t st);
void launch_shift_step(const DevSystem& s, const PanelDev& p, cudaStream_t st);
void launch_full_update(const DevSystem& s, const PanelDev& p, cudaStream_t st);
void launch_full_output(const PanelDev& p, const int32_t* orb2pad, int n_orb, int R, int ncols,
                        int c0, double2* out, cudaStream_t st);
void launch_green_output(const PanelDev& p, int ncols, const int64_t* out_off, double2* out,
                         cudaStream_t st);
void launch_green_deriv_output(const PanelDev& p, int ncols, const int64_t* out_off, double2* out,
                               cudaStream_t st);
void launch_band_energy_terms(const double2* G, const double2* dG, const double* S_el, int64_t n, int K,
                              const double2* z, const double2* w, double g_s, double* e_terms, double* gH,
                              double* gS, cudaStream_t st);
void launch_sum_fixed(const double* v, int64_t n, double* out, cudaStream_t st);
void launch_fma_peak(int mode, int blocks, int threads, int iters, float* out32, double* out64, cudaStream_t st);
// charge-self-consistent forces: per-element gradients at fixed dq, and the Coulomb-gradient term
void launch_csc_force_terms(const double2* G, int64_t n, int K, const double2* z, const double2* w, double g_s,
                            const double* V, const int32_t* atom_a, const int32_t* atom_b, double* gH, double* gS,
                            cudaStream_t st);
void launch_csc_force_coulomb(int n, const double* dgamma, const double* dq, double* F, cudaStream_t st);
void launch_force_blocks(int n_atoms, const int* brow, const int* bcol, const int64_t* boff, const int64_t* ooff,
                         const double* gH, const double* gS, const double* dS_dd, const double* dH_dd,
                         const double* eps, double K, int64_t nvals, double* vblk, cudaStream_t st);
void launch_force_atoms(int n_atoms, const int* brow, const int* bcol, const int64_t* btrans, const double* vblk,
                        double* F, cudaStream_t st);
void launch_mulliken_output(const PanelDev& p, int ncols, const double2* w, double g_s, double* out,
                            cudaStream_t st);

// ragged batches: results of one system's solve into the caller's layout
void launch_scatter_full(const double2* tmp, const int32_t* pos, int K, int Rq, int64_t Nq, int R, int64_t N,
                         int64_t orb0, double2* out, cudaStream_t st);
void launch_scatter_rows(const double2* tmp, const int64_t* gidx, int64_t n, int K, double2* out, cudaStream_t st);
void launch_scatter_cols(const double* tmp, const int32_t* pos, int Rq, double* out, cudaStream_t st);
void launch_scatter_values(const double* v, const int64_t* idx, int64_t n, double* out, cudaStream_t st);

// charge self-consistency (Eq. Hap-CSC)
void launch_csc_potential(const double* gamma, const double* dq, int n, double* V, cudaStream_t st);
void launch_csc_hamiltonian(const DevSystem& s, const double* H0, const double* V, cudaStream_t st);
void launch_atom_sum(const double* q_orb, const int64_t* orb_off, int n_atoms, double* q_atom, cudaStream_t st);
void launch_csc_mix(const double* q, const double* q_ref, const double* dq_in, double* dq_next, double mix, int n,
                    unsigned long long* res_bits, cudaStream_t st);

void launch_lanczos_green(const double* a, const double* b, const double* norm, int R, int n_steps, int K,
                          const double2* z, double2* G, cudaStream_t st);

// generalized Lanczos on a panel of P independent columns (Section 3.2)
void launch_lz_spmv(const DevSystem& s, const double* M, const double2* x, double2* y, int P, cudaStream_t st);
void launch_lz_dot(const PanelDev& p, const double2* x, const double2* y, double* out, int stride, int mode,
                   cudaStream_t st);
void launch_lz_combine(const PanelDev& p, const double2* y, double2* u, double2* u_prev, double2* w,
                       const double* a, const double* b, int sa, int sb, cudaStream_t st);
void launch_lz_scale(const PanelDev& p, double2* w, double2* u, double2* u_prev, const double* bnext, int sb,
                     cudaStream_t st);
void launch_lz_start(const PanelDev& p, const double2* v, double2* u, double* nrm2, cudaStream_t st);

}  // namespace tb
