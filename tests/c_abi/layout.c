/*
 * Prints the size and the field offsets of every struct of the C ABI, one
 * "struct field offset" line per field and "struct sizeof size" per struct,
 * for the comparison with the ctypes mirrors of the Python binding.
 */
#include <stddef.h>
#include <stdio.h>

#include "tbcocg.h"

#define F(S, f) printf(#S " " #f " %zu\n", offsetof(S, f))
#define Z(S) printf(#S " sizeof %zu\n", sizeof(S))

int main(void) {
    Z(tb_system_desc);
    F(tb_system_desc, n_atoms); F(tb_system_desc, orb_per_atom); F(tb_system_desc, brow_ptr);
    F(tb_system_desc, bcol); F(tb_system_desc, S_vals); F(tb_system_desc, H_vals); F(tb_system_desc, eps);
    F(tb_system_desc, K); F(tb_system_desc, precision);
    Z(tb_solve_opts);
    F(tb_solve_opts, tol); F(tb_solve_opts, inner_tol); F(tb_solve_opts, max_iter); F(tb_solve_opts, inner_max_iter);
    F(tb_solve_opts, panel); F(tb_solve_opts, seed); F(tb_solve_opts, switching); F(tb_solve_opts, force_switch_every);
    F(tb_solve_opts, precision); F(tb_solve_opts, inner_lo_tol); F(tb_solve_opts, inner_method);
    F(tb_solve_opts, state_bytes);
    Z(tb_stats);
    F(tb_stats, conv_iter); F(tb_stats, outer_iterations); F(tb_stats, inner_iterations);
    F(tb_stats, max_column_iterations); F(tb_stats, switches); F(tb_stats, unconverged); F(tb_stats, seconds);
    F(tb_stats, inner_redos);
    Z(tb_tune);
    F(tb_tune, panel); F(tb_tune, streams); F(tb_tune, cheb_cpt); F(tb_tune, ctas_per_sm); F(tb_tune, rate);
    Z(tb_csc_opts);
    F(tb_csc_opts, max_scf); F(tb_csc_opts, scf_tol); F(tb_csc_opts, mix);
    Z(tb_csc_stats);
    F(tb_csc_stats, iterations); F(tb_csc_stats, residual); F(tb_csc_stats, outer_iterations);
    F(tb_csc_stats, inner_iterations); F(tb_csc_stats, seconds);
    return 0;
}
