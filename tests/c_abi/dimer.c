/*
 * A C program against the C ABI (include/tbcocg.h): a two-atom s-orbital
 * dimer with overlap s, H by Eq. Hap-1 (H_01 = K eps s).
 *  - host-only calls: the spectrum bounds of S (eigenvalues 1 - s, 1 + s)
 *    and the Chebyshev plan;
 *  - with a device: the Mulliken populations of both orbitals on a line of
 *    shifts against the closed form.  The generalized eigenvalues are
 *    (eps +- h) / (1 +- s); each eigenstate puts half of its occupation on
 *    each orbital, so q_0 = q_1 = g_s / 2 (f(e+) + f(e-)) with the
 *    quadrature's occupation f(e) = -(1/pi) Im sum_k w_k / (z_k - e).
 * Prints "no-device" (exit 0) without a GPU, "ok" (exit 0) when the solve
 * matches, a message and exit 1 otherwise.
 */
#include <complex.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include "tbcocg.h"

#define NK 32

int main(void) {
    const double s = 0.35, eps = -13.6, Kc = 1.75, g_s = 2.0;
    const int32_t opa[2] = {1, 1};
    const int64_t brow[3] = {0, 2, 4};
    const int32_t bcol[4] = {0, 1, 0, 1};
    const double S[4] = {1.0, s, s, 1.0};
    const double e2[2] = {eps, eps};
    tb_system_desc d;
    memset(&d, 0, sizeof(d));
    d.n_atoms = 2;
    d.orb_per_atom = opa;
    d.brow_ptr = brow;
    d.bcol = bcol;
    d.S_vals = S;
    d.H_vals = NULL;
    d.eps = e2;
    d.K = Kc;
    d.precision = TB_FP64;

    double lo = 0.0, hi = 0.0;
    tb_status st = tb_overlap_bounds_desc(&d, &lo, &hi);
    if (st != TB_OK || !(lo > 0.0 && lo <= 1.0 - s && hi >= 1.0 + s)) {
        printf("bounds: %s %g %g\n", tb_status_string(st), lo, hi);
        return 1;
    }
    int32_t n = 0, n_last = 0, rounds = 0;
    double gamma = 0.0;
    float omega[64];
    st = tb_chebyshev_plan(lo, hi, 1e-6, 1e-12, 1000, &n, &n_last, &rounds, &gamma, omega, 64);
    if (st != TB_OK || n < 1 || (n % 2) != 1 || rounds != 2) {
        printf("plan: %s n=%d rounds=%d\n", tb_status_string(st), n, rounds);
        return 1;
    }

    tb_handle *h = NULL;
    st = tb_create(&h, &d, NULL);
    if (st == TB_ERR_NO_DEVICE) {
        printf("no-device\n");
        return 0;
    }
    if (st != TB_OK) {
        printf("tb_create: %s\n", tb_status_string(st));
        return 1;
    }
    /* shifts E_k + 0.5i on [-30, 5] eV with trapezoid weights */
    double z[2 * NK], w[2 * NK];
    for (int k = 0; k < NK; ++k) {
        const double dx = 35.0 / (NK - 1);
        z[2 * k] = -30.0 + k * dx;
        z[2 * k + 1] = 0.5;
        w[2 * k] = (k == 0 || k == NK - 1) ? 0.5 * dx : dx;
        w[2 * k + 1] = 0.0;
    }
    tb_solve_opts o;
    tb_default_opts(&o);
    const int32_t cols[2] = {0, 1};
    double q[2] = {0.0, 0.0};
    st = tb_mulliken_orbital(h, NK, z, w, g_s, 2, cols, &o, q, NULL, NULL);
    tb_destroy(h);
    if (st != TB_OK) {
        printf("tb_mulliken_orbital: %s\n", tb_status_string(st));
        return 1;
    }
    const double hb = Kc * eps * s;
    const double ev[2] = {(eps + hb) / (1.0 + s), (eps - hb) / (1.0 - s)};
    double ref = 0.0;
    for (int m = 0; m < 2; ++m) {
        double complex acc = 0.0;
        for (int k = 0; k < NK; ++k) acc += w[2 * k] / ((z[2 * k] + I * z[2 * k + 1]) - ev[m]);
        ref += -cimag(acc) / 3.14159265358979323846;
    }
    ref *= 0.5 * g_s;
    for (int c = 0; c < 2; ++c)
        if (!(fabs(q[c] - ref) <= 1e-8 * fabs(ref))) {
            printf("q[%d] = %.15g, closed form %.15g\n", c, q[c], ref);
            return 1;
        }
    printf("ok\n");
    return 0;
}
