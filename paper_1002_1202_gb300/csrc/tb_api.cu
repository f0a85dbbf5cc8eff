// C ABI of the generalized shifted COCG library: validation, device memory,
// and the host-side step loop that enqueues the kernels of tb_kernels.cu.
#include "../../include/tbcocg.h"
#include "tb_internal.h"

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <thread>
#include <vector>

using namespace tb;

// Fixed scratch of tb_generalized_lanczos_noalloc: one file-scope device
// array.  Host code must not use the symbol as an address; tb_create asks
// the runtime for the array's device address on the handle's device (which
// also loads the array there: with lazy module loading a module and its
// device arrays are placed on a device only when first used) and keeps it
// in the handle.  From then on the array stays on that GPU until exit.
static __device__ __align__(256) unsigned char g_noalloc_scratch[TB_NOALLOC_SCRATCH_BYTES];

namespace tb {
int max_grid();
}

struct tb_handle {
    DevSystem ds;
    int device = 0;
    int n_atoms = 0;
    int64_t n_orb = 0;
    std::vector<int32_t> orb_per_atom;
    std::vector<int32_t> orb2pad_h;   // caller orbital -> padded slot
    int32_t* orb2pad = nullptr;       // device copy
    double* eps_pad = nullptr;
    int* flags_host = nullptr;        // pinned, NFLAGS ints
    int64_t* atom_orb_off = nullptr;  // device [n_atoms + 1]: first caller orbital of every atom
    double* H0 = nullptr;             // device [nb][16]: the Hamiltonian of tb_create, kept once
                                      // the charge-self-consistent term first replaces H
    // host copies of the caller's pattern and S values (gradient outputs
    // use the caller's block layout)
    std::vector<int64_t> brow_h;       // [n_atoms + 1]
    std::vector<int32_t> bcol_h;       // [nb]
    std::vector<int64_t> boff_h;       // [nb + 1]: first value of every block
    std::vector<int64_t> btrans_h;     // [nb]: index of the transposed block
    std::vector<double> S_h;           // [boff_h[nb]]
    bool ased = false;                 // H built by Eq. Hap-1 from eps and K
    double K = 0.0;
    std::vector<double> eps_h;         // [N] caller order (Eq. Hap-1 handles)
    std::vector<int64_t> sys_atom_off;  // batch: first atom of every system, [n_systems + 1]
    std::vector<int64_t> sys_orb_off;   // batch: first orbital of every system
    // batch only: one solve view per system (block rows offset to the
    // system's first atom, block columns local to it)
    std::vector<DevSystem> sys_ds;
    std::vector<int32_t> orb2pad_local_h;  // [N]: padded slot within the orbital's own system
    int32_t* orb2pad_local = nullptr;      // device copy
    int32_t* bcol_local = nullptr;         // device [nb]: block column local to its system
    int* row_order_local = nullptr;        // device [n_atoms]: per system, its block-row order (local indices)
    int* flags_pool = nullptr;             // pinned [NPOOL][NFLAGS]: status words of the worker threads
    // tb_autotune's choices, per size class (precision, correction method,
    // shift count rounded up to a power of two)
    struct Tuned {
        int prec, method, kb;
        int panel, streams, cpt;
        double rate;
    };
    std::mutex tune_mu;
    std::vector<Tuned> tuned;
    // spectrum of S (Chebyshev corrections of TB_MIXED): bounds [s_lo, s_hi]
    // from a Lanczos run on the host, computed once on first use
    std::once_flag s_once;
    double s_lo = 0.0, s_hi = 0.0;
    tb_status s_status = TB_OK;
    // device address of the allocation-free call's fixed scratch on this
    // handle's device (looked up by tb_create)
    unsigned char* noalloc_base = nullptr;
};

// Device address of g_noalloc_scratch on device dev (which must be current),
// looked up once per device and cached.  The lookup loads the array (and the
// kernels of the allocation-free path, see preload_noalloc_kernels) onto the
// device, so it runs inside tb_create, which allocates anyway.
static tb_status noalloc_scratch(int dev, unsigned char** out) {
    static std::mutex mu;
    static void* addr[256] = {nullptr};
    if (dev < 0 || dev >= 256) return TB_ERR_CUDA;
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return TB_ERR_CUDA;
        }
        if (!preload_noalloc_kernels()) {
            cudaGetLastError();
            return TB_ERR_CUDA;
        }
        addr[dev] = p;
    }
    *out = static_cast<unsigned char*>(addr[dev]);
    return TB_OK;
}

namespace {

struct Cleanup {
    std::vector<void*> dev;
    cudaStream_t st = nullptr;
    void* add(void* p) { dev.push_back(p); return p; }
    ~Cleanup() {
        for (void* p : dev)
            if (p) cudaFreeAsync(p, st);
    }
};

#define TB_CK(call)                                         \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) {                            \
            cudaGetLastError();                             \
            return e_ == cudaErrorMemoryAllocation ? TB_ERR_OOM : TB_ERR_CUDA; \
        }                                                   \
    } while (0)

template <class T>
tb_status dalloc(Cleanup& cl, T** p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    void* q = nullptr;
    cudaError_t e = cudaMallocAsync(&q, count * sizeof(T), cl.st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? TB_ERR_OOM : TB_ERR_CUDA;
    }
    cl.add(q);
    *p = static_cast<T*>(q);
    return TB_OK;
}

bool is_device_ptr(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int next_pow2(int v) {
    int p = 1;
    while (p < v) p <<= 1;
    return p;
}

struct Solve {
    int K = 0;
    const double* z = nullptr;  // host, interleaved
    int R = 0;
    const int32_t* cols = nullptr;
    int proj = PROJ_NONE;
    const int64_t* row_ptr = nullptr;   // PROJ_ROWS
    const int32_t* rows = nullptr;
    const double* w = nullptr;          // PROJ_SROW quadrature weights (host)
    double g_s = 2.0;
    // device outputs
    double2* x_out = nullptr;           // full
    double2* g_out = nullptr;           // rows
    double2* dg_out = nullptr;          // rows: d/dz of the elements (optional)
    const double* rhs = nullptr;        // device [R][N] real right-hand sides (caller order) instead
                                        // of e_j; whole-system views only
    double* q_out = nullptr;            // srow, per column
    // launch choices (0: the handle's tuned value, else the default)
    int streams = 0;                    // panels in flight
    int cheb_cpt = 0;                   // columns per thread of the Chebyshev step
};

// What one solve sees of a system: the device arrays (a whole handle, or one
// system of a batch with block-row pointers offset to its first atom and
// block columns local to it), the caller-orbital -> padded-slot map of its
// orbitals, and a pinned word array for the device status flags.
struct View {
    DevSystem ds;
    const int32_t* o2p_h = nullptr;   // host [n_orb]
    const int32_t* o2p_d = nullptr;   // device [n_orb]
    int64_t n_orb = 0;
    int* flags_host = nullptr;        // pinned [NFLAGS]
    tb_handle* owner = nullptr;       // the handle the view belongs to
};

tb_status check_opts(const tb_solve_opts* o) {
    if (!o) return TB_ERR_INVALID_ARG;
    if (!(o->tol > 0.0) || !(o->inner_tol > 0.0) || o->max_iter < 1 || o->inner_max_iter < 1) return TB_ERR_INVALID_ARG;
    if (o->panel < 0 || o->panel > MAX_P || (o->panel & (o->panel - 1)) != 0) return TB_ERR_INVALID_ARG;
    if (o->seed < 0 || o->force_switch_every < 0) return TB_ERR_INVALID_ARG;
    if (o->precision != TB_FP64 && o->precision != TB_MIXED) return TB_ERR_INVALID_ARG;
    if (o->precision == TB_MIXED && !(o->inner_lo_tol > 0.0 && o->inner_lo_tol < 1.0)) return TB_ERR_INVALID_ARG;
    if (o->inner_method != TB_INNER_CHEBYSHEV && o->inner_method != TB_INNER_CG) return TB_ERR_INVALID_ARG;
    if (o->state_bytes < 0) return TB_ERR_INVALID_ARG;
    return TB_OK;
}

// Device bytes allowed for the full-vector shift state of a call
// (tb_solve_opts::state_bytes; 0 = 8 GiB).
int64_t state_budget(const tb_solve_opts* o) { return o->state_bytes > 0 ? o->state_bytes : (int64_t)8 << 30; }

// The options of one chunk of shifts [k0, k0 + kc): the seed is opts->seed
// when it lies inside the chunk, else the chunk's first shift.
tb_solve_opts chunk_opts(const tb_solve_opts* o, int k0, int kc) {
    tb_solve_opts c = *o;
    c.seed = (o->seed >= k0 && o->seed < k0 + kc) ? o->seed - k0 : 0;
    return c;
}

// ---- spectrum of S for the Chebyshev corrections ---------------------------
// m Lanczos steps on S (FP64, the caller's blocks, no reorthogonalisation:
// the extreme Ritz values are what is wanted, and lost orthogonality only
// repeats converged ones), then the extreme eigenvalues theta of the
// tridiagonal T by Sturm-count bisection and their residual norms
// beta_m |y_m| (y the unit eigenvector of T, by inverse iteration).  Every
// eigenvalue of S lies at or above lambda_min <= theta_min, and some
// eigenvalue lies within the residual of each theta; the bounds widen both
// by their residuals and by a relative margin.  A wrong bound costs
// refinement rounds, never accuracy: the FP64 residual of every round
// decides convergence.
static uint64_t splitmix64(uint64_t& x) {
    uint64_t z = (x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static int sturm_below(const std::vector<double>& a, const std::vector<double>& b, double x) {
    int cnt = 0;
    double d = 1.0;
    for (size_t i = 0; i < a.size(); ++i) {
        d = a[i] - x - (i > 0 ? b[i - 1] * b[i - 1] / d : 0.0);
        if (d == 0.0) d = -1e-300;
        if (d < 0.0) ++cnt;
    }
    return cnt;
}

// k-th smallest eigenvalue (0-based) of the symmetric tridiagonal (a, b)
static double tri_eig(const std::vector<double>& a, const std::vector<double>& b, int k) {
    const size_t m = a.size();
    double lo = a[0], hi = a[0];
    for (size_t i = 0; i < m; ++i) {
        const double r = (i > 0 ? std::fabs(b[i - 1]) : 0.0) + (i + 1 < m ? std::fabs(b[i]) : 0.0);
        lo = std::min(lo, a[i] - r);
        hi = std::max(hi, a[i] + r);
    }
    for (int it = 0; it < 200 && hi - lo > 1e-15 * std::max(1.0, std::fabs(lo) + std::fabs(hi)); ++it) {
        const double mid = 0.5 * (lo + hi);
        if (sturm_below(a, b, mid) > k) hi = mid;
        else lo = mid;
    }
    return 0.5 * (lo + hi);
}

// |last component| of the unit eigenvector of (a, b) for eigenvalue theta
static double tri_last_component(const std::vector<double>& a, const std::vector<double>& b, double theta) {
    const size_t m = a.size();
    const double shift = theta + 1e-10 * (std::fabs(theta) + 1.0);
    std::vector<double> y(m, 1.0), c(m), d(m);
    for (int pass = 0; pass < 3; ++pass) {
        // (T - shift) y_new = y by elimination without pivoting (tiny pivots
        // replaced: only the direction of the result matters)
        for (size_t i = 0; i < m; ++i) {
            double piv = a[i] - shift - (i > 0 ? b[i - 1] * c[i - 1] : 0.0);
            if (std::fabs(piv) < 1e-300) piv = 1e-300;
            c[i] = i + 1 < m ? b[i] / piv : 0.0;
            d[i] = (y[i] - (i > 0 ? b[i - 1] * d[i - 1] : 0.0)) / piv;
        }
        for (size_t i = m; i-- > 0;) y[i] = d[i] - (i + 1 < m ? c[i] * y[i + 1] : 0.0);
        double nrm = 0.0;
        for (double v : y) nrm += v * v;
        nrm = std::sqrt(nrm);
        if (!(nrm > 0.0) || !std::isfinite(nrm)) return 1.0;
        for (double& v : y) v /= nrm;
    }
    return std::fabs(y[m - 1]);
}

// Bounds of the spectrum of a block-sparse symmetric S (caller layout:
// atom block rows brow, block columns bcol, block value offsets boff,
// row-major blocks) by the Lanczos run above.
static tb_status lanczos_bounds(int n, const int32_t* opa, const int64_t* brow, const int32_t* bcol,
                                const int64_t* boff, const double* S, double& lo_out, double& hi_out) {
    std::vector<int64_t> ooff(n + 1, 0);
    for (int i = 0; i < n; ++i) ooff[i + 1] = ooff[i] + opa[i];
    const int64_t N = ooff[n];
    // y = S x, block rows split over host threads for large systems (every
    // row is computed the same way whatever the split)
    const int nthreads = n >= 8192 ? (int)std::max(1u, std::min(16u, std::thread::hardware_concurrency())) : 1;
    auto smul_rows = [&](const std::vector<double>& x, std::vector<double>& y, int I0, int I1) {
        for (int I = I0; I < I1; ++I) {
            const int ni = opa[I];
            double acc[4] = {0.0, 0.0, 0.0, 0.0};
            for (int64_t blk = brow[I]; blk < brow[I + 1]; ++blk) {
                const int J = bcol[blk];
                const int nj = opa[J];
                const double* sb = S + boff[blk];
                for (int a = 0; a < ni; ++a)
                    for (int bj = 0; bj < nj; ++bj) acc[a] += sb[a * nj + bj] * x[ooff[J] + bj];
            }
            for (int a = 0; a < ni; ++a) y[ooff[I] + a] = acc[a];
        }
    };
    auto smul = [&](const std::vector<double>& x, std::vector<double>& y) {
        if (nthreads <= 1) {
            smul_rows(x, y, 0, n);
            return;
        }
        std::vector<std::thread> pool;
        const int chunk = (n + nthreads - 1) / nthreads;
        for (int t = 0; t < nthreads; ++t) {
            const int I0 = t * chunk, I1 = std::min(n, I0 + chunk);
            if (I0 < I1) pool.emplace_back(smul_rows, std::cref(x), std::ref(y), I0, I1);
        }
        for (auto& th : pool) th.join();
    };
    const int m_max = (int)std::min<int64_t>(N, 80);
    std::vector<double> q(N), qp(N, 0.0), w(N), al, be;
    uint64_t seed = 0x5EED5EEDull;
    double nrm = 0.0;
    for (int64_t i = 0; i < N; ++i) {
        q[i] = (double)(splitmix64(seed) >> 11) * 0x1.0p-53 - 0.5;
        nrm += q[i] * q[i];
    }
    nrm = std::sqrt(nrm);
    for (double& v : q) v /= nrm;
    double beta = 0.0, amax = 0.0;
    for (int j = 0; j < m_max; ++j) {
        smul(q, w);
        double a = 0.0;
        for (int64_t i = 0; i < N; ++i) {
            w[i] -= beta * qp[i];
            a += q[i] * w[i];
        }
        double b2 = 0.0;
        for (int64_t i = 0; i < N; ++i) {
            w[i] -= a * q[i];
            b2 += w[i] * w[i];
        }
        beta = std::sqrt(b2);
        al.push_back(a);
        be.push_back(beta);
        amax = std::max(amax, std::fabs(a));
        if (!std::isfinite(beta) || beta <= 1e-12 * amax) break;   // invariant subspace
        for (int64_t i = 0; i < N; ++i) {
            qp[i] = q[i];
            q[i] = w[i] / beta;
        }
    }
    const int m = (int)al.size();
    std::vector<double> boffd(be.begin(), be.end() - 1);
    const double tmin = tri_eig(al, boffd, 0), tmax = tri_eig(al, boffd, m - 1);
    const double bm = be.back();
    const double rmin = bm * tri_last_component(al, boffd, tmin);
    const double rmax = bm * tri_last_component(al, boffd, tmax);
    if (!std::isfinite(tmin) || !std::isfinite(tmax)) return TB_ERR_INVALID_ARG;
    if (!(tmin > 0.0)) return TB_ERR_S_NOT_SPD;
    lo_out = 0.97 * (tmin - rmin);     // <= 0: no usable lower bound, the FP32 CG is used
    hi_out = 1.01 * (tmax + rmax);
    return TB_OK;
}

static void compute_s_bounds(tb_handle* h) {
    h->s_status = lanczos_bounds(h->n_atoms, h->orb_per_atom.data(), h->brow_h.data(), h->bcol_h.data(),
                                 h->boff_h.data(), h->S_h.data(), h->s_lo, h->s_hi);
}

tb_status s_bounds(tb_handle* h, double& lo, double& hi) {
    std::call_once(h->s_once, compute_s_bounds, h);
    lo = h->s_lo;
    hi = h->s_hi;
    return h->s_status;
}

// Coefficients of the Chebyshev corrections: n steps (odd, so that d_n ends
// in x32) reduce the error by at least 1 / T_n(1 / sigma) <= lo_tol per
// round.  R rounds are planned so that lo_tol^(R-1) times the last round's
// reduction reaches inner_tol; the last one needs only that remainder
// (with a factor 2 to spare) and takes n_last <= n steps.  The recurrence
// coefficients do not depend on where it stops, so both share omega.
// A column can end the planned rounds above inner_tol although its true
// residual is below: the double-float residual carries S and x to ~48 bits,
// so its own error is ~2^-47 |S| |x|, which on a cracked Si slab (lambda_min
// of S 0.146, |x| up to ~7 |b|) is ~2e-13 |b|, above inner_tol = 1e-13.  Such
// a column takes up to SPARE more rounds of n_last steps, each followed by
// the residual with FP64 products (only the columns still open do work), and
// only then the FP32 CG.
struct ChebPlan {
    static constexpr int SPARE = 2;
    int n = 0;                 // 0: FP32 CG corrections
    int n_last = 0;            // steps of round R - 1 and of the spare rounds
    int R = 1;                 // rounds planned
    float gamma = 0.f;
    std::vector<float> omega;  // omega[k] multiplies step k (1 <= k < n)
    int steps(int round) const { return round >= R - 1 ? n_last : n; }
    bool chebyshev(int round) const { return n > 0 && round < R + SPARE; }
    // the residual after this round in FP64 (spare rounds; with FP32 CG
    // corrections, from the third round on)
    bool fp64_residual(int round) const { return round >= (n > 0 ? R : 2); }
};

static int cheb_steps(double sigma, double tol) {
    int n = (int)std::ceil(std::acosh(1.0 / std::min(tol, 0.5)) / std::acosh(1.0 / sigma));
    n = std::max(n, 1);
    return (n & 1) ? n : n + 1;
}

ChebPlan cheb_plan(double lo, double hi, double lo_tol, double inner_tol, int cap) {
    ChebPlan cp;
    if (!(lo > 0.0) || !(hi > lo)) return cp;
    const double sigma = (hi - lo) / (hi + lo);
    const int n = cheb_steps(sigma, lo_tol);
    if (n > cap) return cp;
    cp.n = n;
    cp.R = std::max(1, (int)std::ceil(std::log(inner_tol) / std::log(lo_tol) - 1e-9));
    const double rest = 0.5 * inner_tol / std::pow(lo_tol, cp.R - 1);
    cp.n_last = std::min(n, cheb_steps(sigma, rest));
    cp.gamma = (float)(2.0 / (lo + hi));
    cp.omega.assign(n, 0.f);
    double om = 1.0;
    for (int k = 1; k < n; ++k) {
        om = (k == 1) ? 1.0 / (1.0 - 0.5 * sigma * sigma) : 1.0 / (1.0 - 0.25 * om * sigma * sigma);
        cp.omega[k] = (float)om;
    }
    return cp;
}

// Inner CG for S r' = r on the current panel; one host synchronisation in the
// common case (the number of iterations is predicted from the previous call
// and the surplus launches exit at once).
tb_status inner_cg(View& v, const PanelDev& p, int inner_max, int& pred, int64_t& inner_total, cudaStream_t st) {
    int launched = 0;
    int target = std::min(std::max(pred, 1), inner_max);
    while (true) {
        for (int i = launched; i < target; ++i) {
            launch_inner_spmv(v.ds, p, i, st);
            launch_inner_update(v.ds, p, i, st);
        }
        launched = target;
        TB_CK(cudaGetLastError());
        TB_CK(cudaMemcpyAsync(v.flags_host, p.flags, NFLAGS * sizeof(int), cudaMemcpyDeviceToHost, st));
        TB_CK(cudaStreamSynchronize(st));
        prof_harvest();
        if (v.flags_host[1] == 0) {
            inner_total += v.flags_host[3];
            pred = v.flags_host[3] + 1;
            return TB_OK;
        }
        if (launched >= inner_max) return TB_ERR_NOT_CONVERGED;
        target = std::min(launched + 8, inner_max);
    }
}

// FP32 CG of one refinement round (same prediction scheme as inner_cg).
tb_status inner_cg32(View& v, const PanelDev& p, int inner_max, int& pred, int64_t& inner_total,
                     cudaStream_t st) {
    int launched = 0;
    int target = std::min(std::max(pred, 1), inner_max);
    while (true) {
        for (int i = launched; i < target; ++i) {
            launch_inner32_spmv(v.ds, p, i, st);
            launch_inner32_update(v.ds, p, i, st);
        }
        launched = target;
        TB_CK(cudaGetLastError());
        TB_CK(cudaMemcpyAsync(v.flags_host, p.flags, NFLAGS * sizeof(int), cudaMemcpyDeviceToHost, st));
        TB_CK(cudaStreamSynchronize(st));
        prof_harvest();
        if (v.flags_host[1] == 0) {
            if (v.flags_host[4] > 0) {      // the round had work (flags[3] is this round's count)
                inner_total += v.flags_host[3];
                pred = v.flags_host[3] + 1;
            }
            return TB_OK;
        }
        if (launched >= inner_max) return TB_ERR_NOT_CONVERGED;
        target = std::min(launched + 4, inner_max);
    }
}

// TB_DEBUG=1: the refinement state of the first real columns after a failed round
void debug_inner32(View& v, const PanelDev& p, int round, cudaStream_t st) {
    if (!std::getenv("TB_DEBUG")) return;
    std::vector<InnerState> is(2 * p.P);
    cudaMemcpyAsync(is.data(), p.inner32, sizeof(InnerState) * 2 * p.P, cudaMemcpyDeviceToHost, st);
    cudaStreamSynchronize(st);
    std::fprintf(stderr, "[tb] round %d flags %d %d %d %d %d\n", round, v.flags_host[0], v.flags_host[1],
                 v.flags_host[2], v.flags_host[3], v.flags_host[4]);
    double dbg[8] = {0};
    if (p.dbg) {
        cudaMemcpyAsync(dbg, p.dbg, sizeof(dbg), cudaMemcpyDeviceToHost, st);
        cudaStreamSynchronize(st);
        std::fprintf(stderr, "[tb] breakdown it %g rc %g gam %.6e del %.6e den %.6e b2 %.6e gprev %.6e alpha %.6e\n",
                     dbg[0], dbg[1], dbg[2], dbg[3], dbg[4], dbg[5], dbg[6], dbg[7]);
    }
    for (int i = 0; i < 2 * p.P && i < 8; ++i)
        std::fprintf(stderr, "[tb]   col %d: gprev %.3e alpha %.3e beta %.3e b2 %.3e conv %d skip %d scale %.3e\n",
                     i, is[i].gamma_prev, is[i].alpha, is[i].beta, is[i].bnorm2, is[i].conv, is[i].skip,
                     is[i].scale);
}

// TB_TRACE=1 in the environment prints the progress of every refinement round
static const bool g_trace = std::getenv("TB_TRACE") != nullptr;

// TB_GRAPHS=0 in the environment launches the Chebyshev steps one by one
static const bool g_graphs = [] {
    const char* e = std::getenv("TB_GRAPHS");
    return !(e && std::atoi(e) == 0);
}();

// first_round > 0 continues a solve whose first rounds already ran (their
// residual and right-hand side of the next round in place).  capture: only
// enqueue the planned rounds (Chebyshev rounds, whose steps are launched
// one by one into the caller's capture) and return before the host reads
// the status -- the caller reads it after the captured graph ran.
tb_status mixed_inner(View& v, const PanelDev& p, const double2* b, int inner_max, int& pred32,
                      int& rounds_pred, int64_t& inner_total, const ChebPlan& cp, cudaGraphExec_t* graph,
                      cudaStream_t st, int first_round = 0, bool capture = false) {
    // Chebyshev corrections for the planned and the spare rounds (no host
    // round trip); a solve that needs more rounds than that finishes with
    // FP32 CG
    auto cheb_round = [&](int round) { return cp.chebyshev(round); };
    if (first_round == 0) {
        launch_refine_start(v.ds, p, b, st);
        launch_refine_scale(v.ds, p, b, cheb_round(0) ? cp.gamma : 0.f, st);   // f and d_1
    }
    for (int round = first_round;; ++round) {
        if (cheb_round(round)) {
            const int n = cp.steps(round);
            cudaGraphExec_t* gr = graph && !capture ? &graph[n == cp.n ? 0 : 1] : nullptr;
            if (g_graphs && gr && !*gr && n > 2) cheb_graph_build(v.ds, p, cp.omega.data(), n, cp.gamma, gr);
            if (gr && *gr) {
                cheb_graph_launch(*gr, n - 1, st);
            } else {
                for (int k = 1; k < n; ++k) {
                    const float2* cur = (k & 1) ? p.x32 : p.p32;
                    float2* io = (k & 1) ? p.p32 : p.x32;
                    const int mode = k == n - 1 ? 2 : (k == 1 ? 1 : 0);   // 2: adds d_n to the FP64 solution
                    launch_inner32_cheb(v.ds, p, cur, io, cp.omega[k], cp.gamma, mode, st);
                }
            }
            if (n == 1) launch_refine_add(v.ds, p, st);
            inner_total += n;
        } else {
        tb_status s = inner_cg32(v, p, inner_max, pred32, inner_total, st);
        if (s != TB_OK) return s;
        if (g_trace && p.hist) {
            const size_t nh = (size_t)HIST_IT * 2 * p.P * 4;
            std::vector<double> hv(nh);
            cudaMemcpyAsync(hv.data(), p.hist, sizeof(double) * nh, cudaMemcpyDeviceToHost, st);
            cudaStreamSynchronize(st);
            for (int rc = 0; rc < 2 * p.P; ++rc) {
                const double g0 = hv[((size_t)0 * 2 * p.P + rc) * 4];
                double gmax = 0.0;
                int itmax = 0;
                for (int it = 0; it < HIST_IT; ++it) {
                    const double g = hv[((size_t)it * 2 * p.P + rc) * 4];
                    if (g > gmax) { gmax = g; itmax = it; }
                }
                if (g0 > 0.0 && gmax > 10.0 * g0) {
                    std::fprintf(stderr, "[tb] round %d col %d: gamma grows %.3e -> %.3e at it %d\n", round, rc, g0,
                                 gmax, itmax);
                    for (int it = 0; it < 30; ++it) {
                        const double* e = &hv[((size_t)it * 2 * p.P + rc) * 4];
                        std::fprintf(stderr, "[tb]     it %2d gam %.6e del %.6e alpha %.6e beta %.6e\n", it, e[0], e[1],
                                     e[2], e[3]);
                    }
                }
            }
            cudaMemsetAsync(p.hist, 0, sizeof(double) * nh, st);
        }
        if (v.flags_host[0] & (ERR_NOT_SPD | ERR_INNER)) {
            debug_inner32(v, p, round, st);
            return (v.flags_host[0] & ERR_NOT_SPD) ? TB_ERR_S_NOT_SPD : TB_ERR_BREAKDOWN;
        }
        if (round > 0 && v.flags_host[4] == 0) {   // the last residual was already within tolerance
            rounds_pred = round;
            return TB_OK;
        }
        launch_refine_add(v.ds, p, st);
        }
        launch_refine_residual(v.ds, p, b, st, cp.fp64_residual(round));
        launch_refine_scale(v.ds, p, p.Rin, cheb_round(round + 1) ? cp.gamma : 0.f, st);
        if (g_trace) {
            cudaMemcpyAsync(v.flags_host, p.flags, NFLAGS * sizeof(int), cudaMemcpyDeviceToHost, st);
            cudaStreamSynchronize(st);
            std::vector<InnerState> is(2 * p.P);
            cudaMemcpyAsync(is.data(), p.inner32, sizeof(InnerState) * 2 * p.P, cudaMemcpyDeviceToHost, st);
            cudaStreamSynchronize(st);
            double smin = 1e300, smax = 0.0;
            for (auto& x : is)
                if (!x.skip) { smin = std::min(smin, x.scale); smax = std::max(smax, x.scale); }
            std::fprintf(stderr, "[tb] round %d: cg iters %d, unconverged real columns %d, early stops %d, "
                         "scale range %.3e .. %.3e\n", round, v.flags_host[3], v.flags_host[4],
                         v.flags_host[5], smin, smax);
        }
        if (round + 1 >= rounds_pred) {
            if (capture) return TB_OK;
            TB_CK(cudaGetLastError());
            TB_CK(cudaMemcpyAsync(v.flags_host, p.flags, NFLAGS * sizeof(int), cudaMemcpyDeviceToHost, st));
            TB_CK(cudaStreamSynchronize(st));
            prof_harvest();
            if (v.flags_host[0] & ERR_INNER) return TB_ERR_BREAKDOWN;
            if (v.flags_host[4] == 0) {
                rounds_pred = round + 1;
                return TB_OK;
            }
        }
        if (round + 1 >= 8) return TB_ERR_NOT_CONVERGED;
    }
}

struct InnerCtx {
    int pred = 64, pred32 = 32, rounds = 2;
    int64_t total = 0;
    int redo = 0;
    ChebPlan cheb;
    bool res_exact = false;   // Rin holds b - S r' of the last solve (double-float refinement residual)
    // the Chebyshev steps of a full and of a last round as graphs, captured
    // on first use for the PanelDev of this context (its buffers stay fixed)
    cudaGraphExec_t cheb_graph[2] = {nullptr, nullptr};
    InnerCtx() = default;
    InnerCtx(const InnerCtx&) = delete;
    InnerCtx& operator=(const InnerCtx&) = delete;
    ~InnerCtx() {
        cheb_graph_destroy(cheb_graph[0]);
        cheb_graph_destroy(cheb_graph[1]);
    }
};

// The Chebyshev plan of a solve's inner corrections (TB_MIXED with
// TB_INNER_CHEBYSHEV and a usable spectrum of S).
tb_status inner_ctx_init(const View& v, const tb_solve_opts* o, InnerCtx& ic) {
    if (o->precision != TB_MIXED || o->inner_method != TB_INNER_CHEBYSHEV || !v.owner) return TB_OK;
    double lo = 0.0, hi = 0.0;
    const tb_status s = s_bounds(v.owner, lo, hi);
    if (s != TB_OK) return s;
    ic.cheb = cheb_plan(lo, hi, o->inner_lo_tol, o->inner_tol, o->inner_max_iter);
    if (ic.cheb.n > 0) ic.rounds = std::max(ic.cheb.R, 1);   // no host check before the planned last round
    return TB_OK;
}

tb_status inner_redo(View& v, const PanelDev& p, const double2* b, int inner_max, InnerCtx& ic, cudaStream_t st);

// first_round > 0: the mixed solve's first rounds already ran (a captured
// outer step) and their status said that more are needed.
tb_status inner_solve(View& v, const PanelDev& p, const double2* b, int inner_max, InnerCtx& ic,
                      cudaStream_t st, int first_round = 0) {
    ic.res_exact = false;
    if (!p.mixed) return inner_cg(v, p, inner_max, ic.pred, ic.total, st);
    tb_status s = mixed_inner(v, p, b, inner_max, ic.pred32, ic.rounds, ic.total, ic.cheb, ic.cheb_graph, st,
                              first_round);
    if (s == TB_OK) ic.res_exact = b == p.Rcur;
    if (s != TB_ERR_BREAKDOWN && s != TB_ERR_NOT_CONVERGED) return s;
    return inner_redo(v, p, b, inner_max, ic, st);
}

tb_status inner_redo(View& v, const PanelDev& p, const double2* b, int inner_max, InnerCtx& ic, cudaStream_t st) {
    ic.res_exact = false;
    ic.cheb.n = 0;   // the rest of this solve uses the FP32 CG corrections
    // The FP32 corrections failed to converge (or produced a non-finite
    // residual): redo this inner solve with the FP64 CG, on the device.
    // flags[0] keeps no trace of the failed attempt, but keeps the outer
    // recurrence's own error bits (a breakdown of a column's COCG is
    // reported as such, not turned into a redo of the inner solve).
    TB_CK(cudaMemcpyAsync(v.flags_host, p.flags, NFLAGS * sizeof(int), cudaMemcpyDeviceToHost, st));
    TB_CK(cudaStreamSynchronize(st));
    const int keep = v.flags_host[0] & ~ERR_INNER;
    TB_CK(cudaMemcpyAsync(p.flags, &keep, sizeof(int), cudaMemcpyHostToDevice, st));
    TB_CK(cudaMemcpyAsync(p.Rin, b, sizeof(double2) * (size_t)p.npad * p.P, cudaMemcpyDeviceToDevice, st));
    const tb_status s = inner_cg(v, p, inner_max, ic.pred, ic.total, st);
    if (s != TB_OK) return s;
    launch_split_panel(p, st);
    TB_CK(cudaGetLastError());
    ++ic.redo;
    return TB_OK;
}

// Device workspace of a panel's inner solves (FP64 CG; with p.mixed the FP32
// CG and refinement buffers too) and of its grid reductions: everything but
// the shift state.  p.P, p.npad, p.grid and p.mixed must be set.
tb_status alloc_inner_workspace(Cleanup& cl, PanelDev& p, cudaStream_t st) {
    const int P = p.P;
    const size_t nv = (size_t)p.npad * P;
    tb_status s;
    double2** vecs[] = {&p.Rcur, &p.Rprev, &p.Rp, &p.W, &p.Rin, &p.Pin, &p.Sin};
    for (double2** v : vecs) {
        if ((s = dalloc(cl, v, nv)) != TB_OK) return s;
    }
    if (p.mixed) {
        float2** v32[] = {&p.r32, &p.p32, &p.s32, &p.w32, &p.x32};
        for (float2** v : v32) {
            if ((s = dalloc(cl, v, nv)) != TB_OK) return s;
            TB_CK(cudaMemsetAsync(*v, 0, sizeof(float2) * nv, st));
        }
        if ((s = dalloc(cl, &p.RpS, nv)) != TB_OK) return s;
        TB_CK(cudaMemsetAsync(p.RpS, 0, sizeof(float4) * nv, st));
        if ((s = dalloc(cl, &p.inner32, 3 * 2 * P)) != TB_OK) return s;
        if ((s = dalloc(cl, &p.acc32, 8 * P)) != TB_OK) return s;
        if ((s = dalloc(cl, &p.cgs, 4 * P)) != TB_OK) return s;
        if ((s = dalloc(cl, &p.cgu, 2 * P)) != TB_OK) return s;
        if ((s = dalloc(cl, &p.ticket32, 1)) != TB_OK) return s;
        TB_CK(cudaMemsetAsync(p.ticket32, 0, sizeof(unsigned), st));
        if ((s = dalloc(cl, &p.dbg, 8)) != TB_OK) return s;
        if (std::getenv("TB_TRACE")) {
            if ((s = dalloc(cl, &p.hist, (size_t)HIST_IT * 2 * P * 4)) != TB_OK) return s;
            TB_CK(cudaMemsetAsync(p.hist, 0, sizeof(double) * HIST_IT * 2 * P * 4, st));
        }
        TB_CK(cudaMemsetAsync(p.dbg, 0, 8 * sizeof(double), st));
    }
    if ((s = dalloc(cl, &p.col, P)) != TB_OK) return s;
    if ((s = dalloc(cl, &p.inner, 2 * P)) != TB_OK) return s;
    if ((s = dalloc(cl, &p.partials, (size_t)p.grid * 4 * P)) != TB_OK) return s;
    if ((s = dalloc(cl, &p.counter, 1 + MAX_GROUPS)) != TB_OK) return s;
    if ((s = dalloc(cl, &p.partials2, (size_t)MAX_GROUPS * 4 * std::max(p.P, 1))) != TB_OK) return s;
    if ((s = dalloc(cl, &p.flags, NFLAGS)) != TB_OK) return s;
    return TB_OK;
}

// TB_STEP_GRAPHS=0 in the environment runs the outer steps launch by launch
static const bool g_step_graphs = [] {
    const char* e = std::getenv("TB_STEP_GRAPHS");
    return !(e && std::atoi(e) == 0);
}();

// One outer step of a panel on the mixed path with Chebyshev corrections as
// a CUDA graph: the end of step n-1 (rho_{n+1}, the shift step with seed
// switching, and in full mode the x^k, p^k update) and step n up to its
// inner solve (the seed SpMM, r_{n+1}, the planned refinement rounds with
// their Chebyshev steps), then the read of the panel's status words into
// pinned host memory.  Every argument of every launch is fixed for the
// panel (the kernels take the step's scalars from device memory), so the
// graph is captured once and replayed each step with one launch and one
// host synchronisation.  Each captured launch has its own event pair inside
// the graph (external event nodes), so kernel classes are timed per launch
// as with direct launches.
struct StepGraph {
    cudaGraphExec_t exec = nullptr;
    GraphProf prof;
    int rounds = 0;          // planned refinement rounds the graph holds
    int64_t inner_steps = 0; // their Chebyshev steps
    bool failed = false;     // capture failed once: launch directly
    StepGraph() = default;
    StepGraph(const StepGraph&) = delete;
    StepGraph& operator=(const StepGraph&) = delete;
    void reset() {
        if (exec) cudaGraphExecDestroy(exec);
        exec = nullptr;
        graph_prof_release(prof);
    }
    ~StepGraph() { reset(); }
};

bool step_graph_build(View& v, PanelDev& p, InnerCtx& ic, int proj, int inner_max, StepGraph& sg) {
    sg.reset();
    cudaStream_t cs;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    cudaGraph_t g = nullptr;
    bool ok = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
        graph_prof_begin(&sg.prof);
        launch_finish(v.ds, p, cs);
        launch_shift_step(v.ds, p, cs);
        if (proj == PROJ_NONE) launch_full_update(v.ds, p, cs);
        launch_outer_spmm(v.ds, p, true, cs);
        launch_outer_update(v.ds, p, cs);
        int pred32 = ic.pred32, rounds = ic.rounds;
        int64_t steps = 0;
        mixed_inner(v, p, p.Rcur, inner_max, pred32, rounds, steps, ic.cheb, nullptr, cs, 0, true);
        cudaMemcpyAsync(v.flags_host, p.flags, NFLAGS * sizeof(int), cudaMemcpyDeviceToHost, cs);
        graph_prof_end();
        ok = cudaStreamEndCapture(cs, &g) == cudaSuccess && g != nullptr;
        sg.inner_steps = steps;
    }
    if (ok) ok = cudaGraphInstantiate(&sg.exec, g, 0) == cudaSuccess;
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    if (!ok) {
        cudaGetLastError();
        sg.reset();
        sg.failed = true;
        return false;
    }
    sg.rounds = ic.rounds;
    return true;
}

tb_status run_view(View& v, const Solve& q, const tb_solve_opts* o, tb_stats* stats, cudaStream_t st) {
    const auto t0 = std::chrono::steady_clock::now();
    const int K = q.K, R = q.R;
    const int npad = v.ds.npad;
    int P = o->panel ? o->panel : 64;
    P = std::min(P, next_pow2(R));
    if (q.proj == PROJ_NONE) {
        // keep the full-mode x^k, p^k within the state budget (the callers
        // chunk the shifts first; a single shift that still does not fit
        // takes narrower panels)
        while (P > 1 && (double)K * npad * P * 32.0 > (double)state_budget(o)) P >>= 1;
    }
    int M = 0;
    if (q.proj == PROJ_ROWS) {
        for (int c = 0; c < R; ++c) M = std::max<int64_t>(M, q.row_ptr[c + 1] - q.row_ptr[c]);
        if (M < 1) M = 1;
    } else if (q.proj == PROJ_SROW) {
        M = 1;
    }
    Cleanup cl;
    cl.st = st;
    PanelDev p;
    p.P = P;
    p.K = K;
    p.npad = npad;
    p.M = M;
    p.proj = q.proj;
    p.grid = max_grid();
    p.tol = o->tol;
    p.inner_tol = o->inner_tol;
    p.switching = o->switching;
    p.force_switch_every = o->force_switch_every;
    p.mixed = o->precision == TB_MIXED ? 1 : 0;
    p.inner_lo_tol = o->inner_lo_tol;
    p.cheb_cpt = q.cheb_cpt;
    const size_t nv = (size_t)npad * P;
    tb_status s;
    if ((s = alloc_inner_workspace(cl, p, st)) != TB_OK) return s;
    if ((s = dalloc(cl, &p.z, K)) != TB_OK) return s;
    if ((s = dalloc(cl, &p.pi, (size_t)P * K)) != TB_OK) return s;
    if ((s = dalloc(cl, &p.pi_prev, (size_t)P * K)) != TB_OK) return s;
    if ((s = dalloc(cl, &p.conv_iter, (size_t)P * K)) != TB_OK) return s;
    if (q.proj == PROJ_NONE) {
        if ((s = dalloc(cl, &p.ak, (size_t)P * K)) != TB_OK) return s;
        if ((s = dalloc(cl, &p.bk, (size_t)P * K)) != TB_OK) return s;
        if ((s = dalloc(cl, &p.ipi, (size_t)P * K)) != TB_OK) return s;
        if ((s = dalloc(cl, &p.X, nv * K)) != TB_OK) return s;
        if ((s = dalloc(cl, &p.Pk, nv * K)) != TB_OK) return s;
    } else {
        if ((s = dalloc(cl, &p.t, (size_t)P * K * M)) != TB_OK) return s;
        if ((s = dalloc(cl, &p.u, (size_t)P * K * M)) != TB_OK) return s;
        if (q.proj == PROJ_ROWS && (s = dalloc(cl, &p.frow, (size_t)P * M)) != TB_OK) return s;
        if (q.proj == PROJ_ROWS && q.dg_out) {
            p.deriv = 1;
            if ((s = dalloc(cl, &p.dt, (size_t)P * K * M)) != TB_OK) return s;
            if ((s = dalloc(cl, &p.du, (size_t)P * K * M)) != TB_OK) return s;
            if ((s = dalloc(cl, &p.dpi, (size_t)P * K)) != TB_OK) return s;
            if ((s = dalloc(cl, &p.dpi_prev, (size_t)P * K)) != TB_OK) return s;
        }
    }
    double2* w_dev = nullptr;
    if (q.proj == PROJ_SROW) {
        if ((s = dalloc(cl, &w_dev, K)) != TB_OK) return s;
        TB_CK(cudaMemcpyAsync(w_dev, q.w, sizeof(double2) * K, cudaMemcpyHostToDevice, st));
    }
    int64_t* off_dev = nullptr;
    if (q.proj == PROJ_ROWS) {
        if ((s = dalloc(cl, &off_dev, (size_t)R + 1)) != TB_OK) return s;
        TB_CK(cudaMemcpyAsync(off_dev, q.row_ptr, sizeof(int64_t) * (R + 1), cudaMemcpyHostToDevice, st));
    }
    TB_CK(cudaMemcpyAsync(p.z, q.z, sizeof(double2) * K, cudaMemcpyHostToDevice, st));
    TB_CK(cudaMemsetAsync(p.counter, 0, sizeof(unsigned) * (1 + MAX_GROUPS), st));

    std::vector<ColState> colh(P);
    std::vector<int32_t> convh((size_t)P * K);
    std::vector<int32_t> frowh((size_t)P * std::max(M, 1));
    int64_t outer_total = 0, max_col_iters = 0;
    int switches = 0, unconverged = 0, errbits = 0;
    InnerCtx ic;
    if ((s = inner_ctx_init(v, o, ic)) != TB_OK) return s;
    StepGraph sg;
    tb_status final_status = TB_OK;

    for (int c0 = 0; c0 < R; c0 += P) {
        const int ncols = std::min(P, R - c0);
        for (int c = 0; c < P; ++c) {
            ColState cs;
            std::memset(&cs, 0, sizeof(cs));
            cs.zs = make_double2(q.z[2 * o->seed], q.z[2 * o->seed + 1]);
            cs.alpha_prev = make_double2(1.0, 0.0);
            cs.beta_prev = make_double2(0.0, 0.0);
            cs.sc_cur = make_double2(1.0, 0.0);
            cs.sc_prev = make_double2(1.0, 0.0);
            cs.seed = o->seed;
            cs.active = c < ncols ? 1 : 0;
            cs.row = c < ncols && !q.rhs ? v.o2p_h[q.cols[c0 + c]] : -1;
            cs.nfun = q.proj == PROJ_ROWS && c < ncols ? (int)(q.row_ptr[c0 + c + 1] - q.row_ptr[c0 + c])
                                                       : (q.proj == PROJ_SROW ? 1 : 0);
            colh[c] = cs;
            if (q.proj == PROJ_ROWS) {
                for (int m = 0; m < M; ++m) {
                    int slot = 0;
                    if (c < ncols && m < cs.nfun) slot = v.o2p_h[q.rows[q.row_ptr[c0 + c] + m]];
                    frowh[(size_t)c * M + m] = slot;
                }
            }
        }
        TB_CK(cudaMemcpyAsync(p.col, colh.data(), sizeof(ColState) * P, cudaMemcpyHostToDevice, st));
        TB_CK(cudaMemsetAsync(p.inner, 0, sizeof(InnerState) * 2 * P, st));
        if (p.mixed) {
            TB_CK(cudaMemsetAsync(p.inner32, 0, sizeof(InnerState) * 3 * 2 * P, st));
            TB_CK(cudaMemsetAsync(p.acc32, 0, sizeof(double) * 8 * P, st));
        }
        TB_CK(cudaMemsetAsync(p.flags, 0, sizeof(int) * NFLAGS, st));
        if (q.proj == PROJ_ROWS)
            TB_CK(cudaMemcpyAsync(p.frow, frowh.data(), sizeof(int32_t) * P * M, cudaMemcpyHostToDevice, st));

        // r_0 = e_j, r'_0 = S^-1 r_0, rho_0, pi = 1, x^k = 0, p^k = r'_0
        launch_panel_init(v.ds, p, st);
        if (q.rhs) launch_panel_rhs(p, q.rhs + (size_t)c0 * v.n_orb, v.o2p_d, (int)v.n_orb, ncols, st);
        if ((s = inner_solve(v, p, p.Rcur, o->inner_max_iter, ic, st)) != TB_OK) return s;
        if (v.flags_host[0] & ERR_NOT_SPD) return TB_ERR_S_NOT_SPD;
        launch_finish(v.ds, p, st);
        launch_shift_init(v.ds, p, st);
        TB_CK(cudaGetLastError());

        // step n: the end of step n-1 (rho, the shift step, full-mode
        // update: the "tail"), the seed SpMM and r_{n+1}, the inner solve;
        // then the host reads how many columns are still active.  On the
        // mixed path with Chebyshev corrections a step after the first is
        // one replay of the panel's step graph.
        int active = ncols;
        bool tail_pending = false;
        for (int n = 0; n < o->max_iter; ++n) {
            const bool use_graph = tail_pending && g_graphs && g_step_graphs && !g_trace && p.mixed &&
                                   ic.cheb.n > 0 && ic.cheb.chebyshev(ic.rounds - 1) && ic.res_exact && !sg.failed;
            if (use_graph && (!sg.exec || sg.rounds != ic.rounds))
                step_graph_build(v, p, ic, q.proj, o->inner_max_iter, sg);
            if (use_graph && sg.exec) {
                graph_prof_launched(sg.prof);
                TB_CK(cudaGraphLaunch(sg.exec, st));
                TB_CK(cudaStreamSynchronize(st));
                prof_harvest();
                ic.total += sg.inner_steps;
                // the planned rounds ran: what the inner solve does after its
                // host check (redo in FP64 after a non-finite residual, more
                // rounds while some real column is above inner_tol)
                if (v.flags_host[0] & ERR_INNER) s = inner_redo(v, p, p.Rcur, o->inner_max_iter, ic, st);
                else if (v.flags_host[4] > 0) s = inner_solve(v, p, p.Rcur, o->inner_max_iter, ic, st, ic.rounds);
                else {
                    ic.res_exact = true;
                    s = TB_OK;
                }
                if (s != TB_OK) return s;
            } else {
                if (tail_pending) {
                    launch_finish(v.ds, p, st);
                    launch_shift_step(v.ds, p, st);
                    if (q.proj == PROJ_NONE) launch_full_update(v.ds, p, st);
                }
                launch_outer_spmm(v.ds, p, ic.res_exact, st);
                launch_outer_update(v.ds, p, st);
                s = inner_solve(v, p, p.Rcur, o->inner_max_iter, ic, st);
                if (s != TB_OK) return s;
            }
            tail_pending = false;
            active = v.flags_host[2];     // columns still active after step n-1
            errbits |= v.flags_host[0];
            if (errbits & ERR_NOT_SPD) return TB_ERR_S_NOT_SPD;
            if (active == 0) break;
            tail_pending = true;
        }
        if (tail_pending) {   // max_iter ran out: the last step's tail
            launch_finish(v.ds, p, st);
            launch_shift_step(v.ds, p, st);
            if (q.proj == PROJ_NONE) launch_full_update(v.ds, p, st);
            TB_CK(cudaGetLastError());
        }
        // outputs of this panel
        if (q.proj == PROJ_NONE)
            launch_full_output(p, v.o2p_d, (int)v.n_orb, R, ncols, c0, q.x_out, st);
        else if (q.proj == PROJ_ROWS) {
            launch_green_output(p, ncols, off_dev + c0, q.g_out, st);
            if (p.deriv) launch_green_deriv_output(p, ncols, off_dev + c0, q.dg_out, st);
        }
        else
            launch_mulliken_output(p, ncols, w_dev, q.g_s, q.q_out + c0, st);
        TB_CK(cudaGetLastError());
        TB_CK(cudaMemcpyAsync(colh.data(), p.col, sizeof(ColState) * P, cudaMemcpyDeviceToHost, st));
        TB_CK(cudaMemcpyAsync(convh.data(), p.conv_iter, sizeof(int32_t) * P * K, cudaMemcpyDeviceToHost, st));
        TB_CK(cudaMemcpyAsync(v.flags_host, p.flags, NFLAGS * sizeof(int), cudaMemcpyDeviceToHost, st));
        TB_CK(cudaStreamSynchronize(st));
        errbits |= v.flags_host[0];
        for (int c = 0; c < ncols; ++c) {
            outer_total += colh[c].iters;
            max_col_iters = std::max<int64_t>(max_col_iters, colh[c].iters);
            switches += colh[c].switches;
            for (int k = 0; k < K; ++k) {
                const int ci = convh[(size_t)c * K + k];
                if (ci < 0) ++unconverged;
                if (stats && stats->conv_iter) stats->conv_iter[(size_t)(c0 + c) * K + k] = ci;
            }
        }
    }
    if (errbits & ERR_NOT_SPD) final_status = TB_ERR_S_NOT_SPD;
    else if (errbits & ERR_BREAKDOWN) final_status = TB_ERR_BREAKDOWN;
    else if (unconverged > 0) final_status = TB_ERR_NOT_CONVERGED;
    if (stats) {
        stats->outer_iterations = outer_total;
        stats->inner_iterations = ic.total;
        stats->max_column_iterations = max_col_iters;
        stats->switches = switches;
        stats->unconverged = unconverged;
        stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        stats->inner_redos = ic.redo;
    }
    return final_status;
}

// The whole handle as one view (a single system, or a batch seen as one
// block-diagonal system).
View whole_view(tb_handle* h) {
    View v;
    v.ds = h->ds;
    v.o2p_h = h->orb2pad_h.data();
    v.o2p_d = h->orb2pad;
    v.n_orb = h->n_orb;
    v.flags_host = h->flags_host;
    v.owner = h;
    return v;
}

// Concurrent jobs: the requested columns are grouped by system (a batch)
// and cut into panel-sized chunks; every chunk is solved on its system's
// view (no work on the rows of other systems) by a pool of host threads,
// each driving its own stream, so that the chunks' kernels overlap on the
// GPU (they fill each other's reduction tails, small kernels and host
// round trips).  Results land in temporary buffers and are scattered into
// the caller's layout; entries that couple two systems of a batch are zero.
tb_status run_jobs(tb_handle* h, const Solve& q, const tb_solve_opts* o, tb_stats* stats, cudaStream_t st,
                   int max_workers) {
    const auto t0 = std::chrono::steady_clock::now();
    const bool batch = !h->sys_ds.empty();
    const int ns = batch ? (int)h->sys_ds.size() : 1;
    const int K = q.K, R = q.R;
    std::vector<std::vector<int>> members(ns);
    for (int c = 0; c < R; ++c) {
        const int sys = batch ? (int)(std::upper_bound(h->sys_orb_off.begin(), h->sys_orb_off.end(),
                                                       (int64_t)q.cols[c]) - h->sys_orb_off.begin()) - 1
                              : 0;
        members[sys].push_back(c);
    }
    if (q.proj == PROJ_NONE)
        TB_CK(cudaMemsetAsync(q.x_out, 0, sizeof(double2) * (size_t)K * R * h->n_orb, st));
    if (q.proj == PROJ_ROWS) {
        TB_CK(cudaMemsetAsync(q.g_out, 0, sizeof(double2) * (size_t)q.row_ptr[R] * K, st));
        if (q.dg_out) TB_CK(cudaMemsetAsync(q.dg_out, 0, sizeof(double2) * (size_t)q.row_ptr[R] * K, st));
    }
    cudaEvent_t ev_in;
    TB_CK(cudaEventCreateWithFlags(&ev_in, cudaEventDisableTiming));
    TB_CK(cudaEventRecord(ev_in, st));
    // chunks of one panel each (the width run_view would pick for the system)
    struct Job {
        int sys;
        std::vector<int> cols;
    };
    std::vector<Job> jobs;
    for (int sys = 0; sys < ns; ++sys) {
        const int Rs = (int)members[sys].size();
        if (Rs == 0) continue;
        int Pw = o->panel ? o->panel : 64;
        Pw = std::min(Pw, next_pow2(Rs));
        for (int c0 = 0; c0 < Rs; c0 += Pw)
            jobs.push_back({sys, std::vector<int>(members[sys].begin() + c0,
                                                  members[sys].begin() + std::min(Rs, c0 + Pw))});
    }
    const int nw = std::min<int>({(int)jobs.size(), max_workers, NPOOL});
    std::atomic<int> next{0};
    std::mutex mu;
    tb_status worst = TB_OK;
    bool unconverged = false;
    tb_stats agg{};
    auto worker = [&](int wid) {
        cudaSetDevice(h->device);
        cudaStream_t ws = nullptr;
        if (cudaStreamCreateWithFlags(&ws, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            std::lock_guard<std::mutex> lk(mu);
            if (worst == TB_OK) worst = TB_ERR_CUDA;
            return;
        }
        cudaStreamWaitEvent(ws, ev_in, 0);
        for (int j = next++; j < (int)jobs.size(); j = next++) {
            const int sys = jobs[j].sys;
            const std::vector<int>& mem = jobs[j].cols;
            const int Rq = (int)mem.size();
            const int64_t orb0 = batch ? h->sys_orb_off[sys] : 0;
            const int64_t Nq = batch ? h->sys_orb_off[sys + 1] - orb0 : h->n_orb;
            tb_status s = TB_OK;
            {
                Cleanup cl;
                cl.st = ws;
                View v = whole_view(h);
                if (batch) {
                    v.ds = h->sys_ds[sys];
                    v.o2p_h = h->orb2pad_local_h.data() + orb0;
                    v.o2p_d = h->orb2pad_local + orb0;
                    v.n_orb = Nq;
                }
                v.flags_host = h->flags_pool + (size_t)NFLAGS * wid;
                std::vector<int32_t> cols(Rq), pos(Rq);
                for (int i = 0; i < Rq; ++i) {
                    pos[i] = mem[i];
                    cols[i] = (int32_t)(q.cols[mem[i]] - orb0);
                }
                Solve q2 = q;
                q2.R = Rq;
                q2.cols = cols.data();
                std::vector<int64_t> rp2, gidx;
                std::vector<int32_t> rows2;
                int32_t* pos_d = nullptr;
                if ((s = dalloc(cl, &pos_d, (size_t)Rq)) == TB_OK &&
                    cudaMemcpyAsync(pos_d, pos.data(), sizeof(int32_t) * Rq, cudaMemcpyHostToDevice, ws) != cudaSuccess)
                    s = TB_ERR_CUDA;
                double2* xt = nullptr;
                double2* gt = nullptr;
                double2* dgt = nullptr;
                double* qt = nullptr;
                int64_t* gidx_d = nullptr;
                if (s == TB_OK && q.proj == PROJ_NONE) {
                    s = dalloc(cl, &xt, (size_t)K * Rq * Nq);
                    q2.x_out = xt;
                } else if (s == TB_OK && q.proj == PROJ_ROWS) {
                    // rows inside the column's system only; the others stay zero
                    rp2.push_back(0);
                    for (int i = 0; i < Rq; ++i) {
                        const int c = mem[i];
                        for (int64_t m = q.row_ptr[c]; m < q.row_ptr[c + 1]; ++m) {
                            const int64_t r = q.rows[m];
                            if (r >= orb0 && r < orb0 + Nq) {
                                rows2.push_back((int32_t)(r - orb0));
                                gidx.push_back(m);
                            }
                        }
                        rp2.push_back((int64_t)rows2.size());
                    }
                    if (rows2.empty()) rows2.push_back(0);   // keep the arrays non-empty
                    q2.row_ptr = rp2.data();
                    q2.rows = rows2.data();
                    if ((s = dalloc(cl, &gt, (size_t)std::max<int64_t>(1, rp2.back()) * K)) == TB_OK &&
                        (s = dalloc(cl, &gidx_d, std::max<size_t>(1, gidx.size()))) == TB_OK && !gidx.empty() &&
                        cudaMemcpyAsync(gidx_d, gidx.data(), sizeof(int64_t) * gidx.size(), cudaMemcpyHostToDevice,
                                        ws) != cudaSuccess)
                        s = TB_ERR_CUDA;
                    q2.g_out = gt;
                    if (s == TB_OK && q.dg_out) s = dalloc(cl, &dgt, (size_t)std::max<int64_t>(1, rp2.back()) * K);
                    q2.dg_out = q.dg_out ? dgt : nullptr;
                } else if (s == TB_OK) {
                    s = dalloc(cl, &qt, (size_t)Rq);
                    q2.q_out = qt;
                }
                tb_stats st2{};
                std::vector<int32_t> conv;
                if (stats && stats->conv_iter) {
                    conv.assign((size_t)Rq * K, -1);
                    st2.conv_iter = conv.data();
                }
                if (s == TB_OK) s = run_view(v, q2, o, &st2, ws);
                if (s == TB_OK || s == TB_ERR_NOT_CONVERGED) {
                    if (q.proj == PROJ_NONE)
                        launch_scatter_full(xt, pos_d, K, Rq, Nq, R, h->n_orb, orb0, q.x_out, ws);
                    else if (q.proj == PROJ_ROWS && !gidx.empty()) {
                        launch_scatter_rows(gt, gidx_d, (int64_t)gidx.size(), K, q.g_out, ws);
                        if (q.dg_out) launch_scatter_rows(dgt, gidx_d, (int64_t)gidx.size(), K, q.dg_out, ws);
                    }
                    else if (q.proj == PROJ_SROW)
                        launch_scatter_cols(qt, pos_d, Rq, q.q_out, ws);
                    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(ws) != cudaSuccess) s = TB_ERR_CUDA;
                }
                std::lock_guard<std::mutex> lk(mu);
                if (s == TB_ERR_NOT_CONVERGED) unconverged = true;
                else if (s != TB_OK && worst == TB_OK) worst = s;
                agg.outer_iterations += st2.outer_iterations;
                agg.inner_iterations += st2.inner_iterations;
                agg.max_column_iterations = std::max(agg.max_column_iterations, st2.max_column_iterations);
                agg.switches += st2.switches;
                agg.unconverged += st2.unconverged;
                agg.inner_redos += st2.inner_redos;
                if (stats && stats->conv_iter)
                    for (int i = 0; i < Rq; ++i)
                        for (int k = 0; k < K; ++k) stats->conv_iter[(size_t)pos[i] * K + k] = conv[(size_t)i * K + k];
            }
            cudaStreamSynchronize(ws);   // the view's temporaries are freed in stream order
        }
        cudaStreamDestroy(ws);
    };
    std::vector<std::thread> pool;
    for (int w = 1; w < nw; ++w) pool.emplace_back(worker, w);
    worker(0);
    for (auto& t : pool) t.join();
    cudaEventDestroy(ev_in);
    if (stats) {
        int32_t* ci = stats->conv_iter;
        *stats = agg;
        stats->conv_iter = ci;
        stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    if (worst != TB_OK) return worst;
    return unconverged ? TB_ERR_NOT_CONVERGED : TB_OK;
}

// Worker threads of one call: up to 8 for a batch (many small systems), 4
// for one system (panels in flight fill each other's reduction tails, small
// kernels and host round trips; measured on a 4096-atom system at 256
// columns per panel: 1.00 / 1.21 / 1.32 / 1.36x the one-panel throughput
// with 1 / 2 / 3 / 4 panels in flight); TB_STREAMS=n overrides (1: one panel
// at a time on the caller's stream).
int workers_for(const tb_handle* h) {
    static const int forced = [] {
        const char* e = std::getenv("TB_STREAMS");
        return e ? std::max(1, std::atoi(e)) : 0;
    }();
    if (forced) return forced;
    return h->sys_ds.empty() ? 4 : 8;
}

// The tuned choices of this handle for a call (nullptr: none).
const tb_handle::Tuned* tuned_for(tb_handle* h, const tb_solve_opts* o, int K) {
    std::lock_guard<std::mutex> lk(h->tune_mu);
    const int kb = next_pow2(K);
    for (const auto& t : h->tuned)
        if (t.prec == o->precision && t.method == o->inner_method && t.kb == kb) return &t;
    return nullptr;
}

tb_status run_solve(tb_handle* h, const Solve& q0, const tb_solve_opts* o, tb_stats* stats, cudaStream_t st) {
    // automatic choices: the handle's tuned panel width, panels in flight and
    // Chebyshev-step form for this size class, else the defaults
    Solve q = q0;
    tb_solve_opts oe = *o;
    const tb_handle::Tuned* t = o->panel == 0 ? tuned_for(h, o, q.K) : nullptr;
    if (t) oe.panel = t->panel;
    if (q.cheb_cpt == 0 && t) q.cheb_cpt = t->cpt;
    const int nw = q.streams ? q.streams : (t ? t->streams : workers_for(h));
    const int Pw = std::min(oe.panel ? oe.panel : 64, next_pow2(q.R));
    if (h->sys_ds.empty() && (nw == 1 || q.R <= Pw)) {
        View v = whole_view(h);
        return run_view(v, q, &oe, stats, st);
    }
    return run_jobs(h, q, &oe, stats, st, nw);
}

tb_status check_cols(const tb_handle* h, int R, const int32_t* cols) {
    if (R < 1 || !cols) return TB_ERR_INVALID_ARG;
    for (int c = 0; c < R; ++c)
        if (cols[c] < 0 || cols[c] >= h->n_orb) return TB_ERR_INVALID_ARG;
    return TB_OK;
}

tb_status check_shifts(int K, const double* z, const tb_solve_opts* o) {
    if (K < 1 || K > MAX_K || !z) return TB_ERR_INVALID_ARG;
    if (o->seed >= K) return TB_ERR_INVALID_ARG;
    for (int k = 0; k < 2 * K; ++k)
        if (!std::isfinite(z[k])) return TB_ERR_INVALID_ARG;
    return TB_OK;
}

// Output staging: write straight into device memory, or into a temporary
// that is copied to the caller's host buffer at the end.
struct OutBuf {
    void* user = nullptr;
    void* dev = nullptr;
    size_t bytes = 0;
    bool host = false;
};

tb_status out_prepare(Cleanup& cl, OutBuf& ob, void* user, size_t bytes) {
    ob.user = user;
    ob.bytes = bytes;
    ob.host = !is_device_ptr(user);
    if (!ob.host) {
        ob.dev = user;
        return TB_OK;
    }
    char* d = nullptr;
    tb_status s = dalloc(cl, &d, bytes);
    ob.dev = d;
    return s;
}

tb_status out_finish(const OutBuf& ob, cudaStream_t st) {
    if (ob.host) TB_CK(cudaMemcpyAsync(ob.user, ob.dev, ob.bytes, cudaMemcpyDeviceToHost, st));
    TB_CK(cudaStreamSynchronize(st));
    return TB_OK;
}

tb_status merge(tb_status run, tb_status fin) { return run != TB_OK && run != TB_ERR_NOT_CONVERGED ? run : (fin != TB_OK ? fin : run); }

// Groups of consecutive atoms for the grouped FP32 SpMV: for each group the
// ascending list of its distinct block columns and, per block, the position
// of its column in that list.  G is 16 or 8 (CTAs of 256 or 128 threads),
// the larger whose shared memory (neighbour-union panel rows of a 32-column
// slice plus the group's S blocks) lets two CTAs share an SM; with neither
// (dense neighbourhoods, e.g. ~39 neighbour atoms in liquid water) the
// register-gather form is faster and no groups are built.
// TB_SPMV_GROUP=G forces G (any of 16, 8, 4, 2; 0 turns the form off).
struct SpmvGroups {
    int G = 0, n_groups = 0, max_union = 0, max_gblocks = 0;
    std::vector<int> ptr, cols, loc;
};

SpmvGroups build_spmv_groups(const std::vector<int>& brow, const std::vector<int>& bcol, int n) {
    const size_t budget = 113 * 1024;
    int forced = -1;
    if (const char* env = std::getenv("TB_SPMV_GROUP")) forced = std::atoi(env);
    SpmvGroups out;
    if (forced == 0) return out;
    for (int G : {16, 8, 4, 2}) {
        if (forced > 0 ? G != forced : G < 8) continue;
        SpmvGroups g;
        g.G = G;
        g.n_groups = (n + G - 1) / G;
        g.ptr.assign(g.n_groups + 1, 0);
        g.loc.assign(bcol.size(), 0);
        std::vector<int> u;
        for (int q = 0; q < g.n_groups; ++q) {
            const int a0 = q * G, a1 = std::min(n, a0 + G);
            u.assign(bcol.begin() + brow[a0], bcol.begin() + brow[a1]);
            std::sort(u.begin(), u.end());
            u.erase(std::unique(u.begin(), u.end()), u.end());
            for (int b = brow[a0]; b < brow[a1]; ++b)
                g.loc[b] = (int)(std::lower_bound(u.begin(), u.end(), bcol[b]) - u.begin());
            g.cols.insert(g.cols.end(), u.begin(), u.end());
            g.ptr[q + 1] = (int)g.cols.size();
            g.max_union = std::max(g.max_union, (int)u.size());
            g.max_gblocks = std::max(g.max_gblocks, brow[a1] - brow[a0]);
        }
        const size_t xregion = (size_t)g.max_union * 4 * 32 * 8;
        const size_t red = (size_t)(G / 2) * 16 * 8 * 8;
        const size_t smem = 128 + std::max(xregion, red) + (size_t)g.max_gblocks * 64;
        if (smem <= budget || (forced > 0 && smem <= 226 * 1024)) return g;
    }
    return out;
}

}  // namespace

namespace {

// Keep the Hamiltonian of tb_create before the first charge-dependent one
// replaces it.
tb_status ensure_H0(tb_handle* h, cudaStream_t st) {
    if (h->H0) return TB_OK;
    const size_t bytes = sizeof(double) * 16 * (size_t)h->ds.nb;
    cudaError_t e = cudaMalloc(&h->H0, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        h->H0 = nullptr;
        return e == cudaErrorMemoryAllocation ? TB_ERR_OOM : TB_ERR_CUDA;
    }
    TB_CK(cudaMemcpyAsync(h->H0, h->ds.H, bytes, cudaMemcpyDeviceToDevice, st));
    return TB_OK;
}

// A device copy of a host-or-device array (device arrays are used in place).
template <class T>
tb_status device_view(Cleanup& cl, const T* src, size_t count, const T** out, cudaStream_t st) {
    if (is_device_ptr(src)) {
        *out = src;
        return TB_OK;
    }
    T* d = nullptr;
    tb_status s = dalloc(cl, &d, count);
    if (s != TB_OK) return s;
    TB_CK(cudaMemcpyAsync(d, src, sizeof(T) * count, cudaMemcpyHostToDevice, st));
    *out = d;
    return TB_OK;
}

}  // namespace

namespace {

// Atomic populations of every atom into the device array q_atom: all N
// orbitals solved (PROJ_SROW) into a device buffer, then summed per atom on
// the device.
tb_status mulliken_atoms_device(tb_handle* h, int32_t K, const double* z, const double* w, double g_s,
                                const tb_solve_opts* opts, double* q_atom, tb_stats* stats, cudaStream_t st) {
    tb_status s;
    if ((s = check_opts(opts)) != TB_OK) return s;
    if ((s = check_shifts(K, z, opts)) != TB_OK) return s;
    if (!w || !std::isfinite(g_s)) return TB_ERR_INVALID_ARG;
    for (int k = 0; k < 2 * K; ++k)
        if (!std::isfinite(w[k])) return TB_ERR_INVALID_ARG;
    std::vector<int32_t> cols(h->n_orb);
    for (int64_t o = 0; o < h->n_orb; ++o) cols[o] = (int32_t)o;
    Cleanup cl;
    cl.st = st;
    double* q_orb = nullptr;
    if ((s = dalloc(cl, &q_orb, (size_t)h->n_orb)) != TB_OK) return s;
    Solve q;
    q.K = K; q.z = z; q.R = (int)h->n_orb; q.cols = cols.data(); q.proj = PROJ_SROW; q.w = w; q.g_s = g_s;
    q.q_out = q_orb;
    const tb_status run = run_solve(h, q, opts, stats, st);
    if (run != TB_OK && run != TB_ERR_NOT_CONVERGED) return run;
    launch_atom_sum(q_orb, h->atom_orb_off, h->n_atoms, q_atom, st);
    TB_CK(cudaGetLastError());
    return run;
}

}  // namespace

extern "C" {

const char* tb_status_string(tb_status s) {
    switch (s) {
        case TB_OK: return "TB_OK";
        case TB_ERR_INVALID_ARG: return "TB_ERR_INVALID_ARG";
        case TB_ERR_NOT_SYMMETRIC: return "TB_ERR_NOT_SYMMETRIC";
        case TB_ERR_S_NOT_SPD: return "TB_ERR_S_NOT_SPD";
        case TB_ERR_OOM: return "TB_ERR_OOM";
        case TB_ERR_CUDA: return "TB_ERR_CUDA";
        case TB_ERR_NOT_CONVERGED: return "TB_ERR_NOT_CONVERGED";
        case TB_ERR_BREAKDOWN: return "TB_ERR_BREAKDOWN";
        case TB_ERR_TIMEOUT: return "TB_ERR_TIMEOUT";
        case TB_ERR_NO_DEVICE: return "TB_ERR_NO_DEVICE";
        case TB_ERR_TOO_LARGE: return "TB_ERR_TOO_LARGE";
    }
    return "TB_UNKNOWN_STATUS";
}

void tb_default_opts(tb_solve_opts* o) {
    if (!o) return;
    o->tol = 1e-10;
    o->inner_tol = 1e-13;
    o->max_iter = 100000;
    o->inner_max_iter = 1000;
    o->panel = 0;
    o->seed = 0;
    o->switching = 1;
    o->force_switch_every = 0;
    o->precision = TB_FP64;
    o->inner_lo_tol = 1e-6;
    o->inner_method = TB_INNER_CHEBYSHEV;
    o->state_bytes = 0;
}

tb_status tb_measure_fma_peak(int32_t mode, double* tflops_out, void* stream) {
    if (!tflops_out || mode < 0 || mode > 2) return TB_ERR_INVALID_ARG;
    int dev = 0, sms = 0;
    TB_CK(cudaGetDevice(&dev));
    TB_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int threads = 256, blocks = 8 * sms;          // 64 warps per SM
    const int iters = mode == 2 ? 1 << 11 : 1 << 13;
    cudaEvent_t e0, e1;
    TB_CK(cudaEventCreate(&e0));
    TB_CK(cudaEventCreate(&e1));
    launch_fma_peak(mode, blocks, threads, iters / 16, nullptr, nullptr, st);   // warm-up
    TB_CK(cudaEventRecord(e0, st));
    launch_fma_peak(mode, blocks, threads, iters, nullptr, nullptr, st);
    TB_CK(cudaEventRecord(e1, st));
    TB_CK(cudaEventSynchronize(e1));
    float ms = 0.f;
    TB_CK(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    // 8 chains x 2 flop per FMA (x 2 lanes for the packed form) per round
    const double flops = (double)blocks * threads * iters * 8 * 2 * (mode == 1 ? 2 : 1);
    *tflops_out = ms > 0.f ? flops / (ms * 1e-3) / 1e12 : 0.0;
    return TB_OK;
}

int64_t tb_launch_count(void) { return launch_count(); }

void tb_profile_enable(int32_t enable) { profile_enable(enable != 0); }

tb_status tb_profile_read(int32_t kernel, int64_t* launches, double* total_ms) {
    if (kernel < 0 || kernel >= K_COUNT || !launches || !total_ms) return TB_ERR_INVALID_ARG;
    profile_read(kernel, launches, total_ms);
    return TB_OK;
}

tb_status tb_profile_busy(int32_t kernel, double* busy_ms) {
    if (kernel < 0 || kernel >= K_COUNT || !busy_ms) return TB_ERR_INVALID_ARG;
    *busy_ms = profile_busy(kernel);
    return TB_OK;
}

int64_t tb_num_orbitals(const tb_handle* h) { return h ? h->n_orb : 0; }
int64_t tb_num_atoms(const tb_handle* h) { return h ? h->n_atoms : 0; }
int64_t tb_num_blocks(const tb_handle* h) { return h ? h->ds.nb : 0; }

tb_status tb_destroy(tb_handle* h) {
    if (!h) return TB_OK;
    cudaFree(h->ds.brow);
    cudaFree(h->ds.bcol);
    cudaFree(h->ds.S);
    cudaFree(h->ds.H);
    cudaFree(h->ds.S32);
    cudaFree(h->ds.S32lo);
    cudaFree(h->ds.S32T);
    cudaFree(h->ds.norb);
    cudaFree(h->ds.row_order);
    cudaFree(h->ds.S32r);
    cudaFree(h->ds.bmeta);
    cudaFree(h->row_order_local);
    cudaFree(h->ds.H32hi);
    cudaFree(h->ds.H32lo);
    cudaFree(h->ds.grp_ptr);
    cudaFree(h->ds.grp_cols);
    cudaFree(h->ds.blk_loc);
    cudaFree(h->orb2pad);
    cudaFree(h->eps_pad);
    cudaFree(h->atom_orb_off);
    cudaFree(h->H0);
    cudaFree(h->orb2pad_local);
    cudaFree(h->bcol_local);
    if (h->flags_pool) cudaFreeHost(h->flags_pool);
    if (h->flags_host) cudaFreeHost(h->flags_host);
    delete h;
    return TB_OK;
}

tb_status tb_create(tb_handle** out, const tb_system_desc* d, void* stream) {
    if (!out) return TB_ERR_INVALID_ARG;
    *out = nullptr;
    if (!d || d->n_atoms < 1 || !d->orb_per_atom || !d->brow_ptr || !d->bcol || !d->S_vals) return TB_ERR_INVALID_ARG;
    if (d->precision != TB_FP64) return TB_ERR_INVALID_ARG;
    if (!d->H_vals && (!d->eps || !std::isfinite(d->K))) return TB_ERR_INVALID_ARG;
    const int n = d->n_atoms;
    if ((int64_t)n * 4 > (int64_t)1 << 30) return TB_ERR_INVALID_ARG;
    // ---- structure ----
    std::vector<int64_t> ooff(n + 1, 0);
    for (int i = 0; i < n; ++i) {
        const int o = d->orb_per_atom[i];
        if (o != 1 && o != 4) return TB_ERR_INVALID_ARG;
        ooff[i + 1] = ooff[i] + o;
    }
    const int64_t N = ooff[n];
    if (d->brow_ptr[0] != 0) return TB_ERR_INVALID_ARG;
    for (int i = 0; i < n; ++i)
        if (d->brow_ptr[i + 1] < d->brow_ptr[i]) return TB_ERR_INVALID_ARG;
    const int64_t nb = d->brow_ptr[n];
    if (nb < n || nb > INT32_MAX) return TB_ERR_INVALID_ARG;
    std::vector<int64_t> boff(nb + 1, 0);
    for (int i = 0; i < n; ++i) {
        bool diag = false;
        for (int64_t b = d->brow_ptr[i]; b < d->brow_ptr[i + 1]; ++b) {
            const int j = d->bcol[b];
            if (j < 0 || j >= n) return TB_ERR_INVALID_ARG;
            if (b > d->brow_ptr[i] && d->bcol[b - 1] >= j) return TB_ERR_INVALID_ARG;
            if (j == i) diag = true;
            boff[b + 1] = boff[b] + (int64_t)d->orb_per_atom[i] * d->orb_per_atom[j];
        }
        if (!diag) return TB_ERR_INVALID_ARG;
    }
    // ---- symmetry of pattern and values ----
    double smax = 0.0, hmax = 0.0;
    for (int64_t e = 0; e < boff[nb]; ++e) {
        if (!std::isfinite(d->S_vals[e])) return TB_ERR_INVALID_ARG;
        smax = std::max(smax, std::fabs(d->S_vals[e]));
        if (d->H_vals) {
            if (!std::isfinite(d->H_vals[e])) return TB_ERR_INVALID_ARG;
            hmax = std::max(hmax, std::fabs(d->H_vals[e]));
        }
    }
    std::vector<int64_t> btrans(nb);
    for (int i = 0; i < n; ++i) {
        const int ni = d->orb_per_atom[i];
        for (int64_t b = d->brow_ptr[i]; b < d->brow_ptr[i + 1]; ++b) {
            const int j = d->bcol[b];
            const int nj = d->orb_per_atom[j];
            const int32_t* beg = d->bcol + d->brow_ptr[j];
            const int32_t* end = d->bcol + d->brow_ptr[j + 1];
            const int32_t* f = std::lower_bound(beg, end, (int32_t)i);
            if (f == end || *f != i) return TB_ERR_NOT_SYMMETRIC;
            const int64_t bt = d->brow_ptr[j] + (f - beg);
            btrans[b] = bt;
            for (int a = 0; a < ni; ++a)
                for (int c = 0; c < nj; ++c) {
                    const double s1 = d->S_vals[boff[b] + (int64_t)a * nj + c];
                    const double s2 = d->S_vals[boff[bt] + (int64_t)c * ni + a];
                    if (std::fabs(s1 - s2) > 1e-12 * smax) return TB_ERR_NOT_SYMMETRIC;
                    if (d->H_vals) {
                        const double h1 = d->H_vals[boff[b] + (int64_t)a * nj + c];
                        const double h2 = d->H_vals[boff[bt] + (int64_t)c * ni + a];
                        if (std::fabs(h1 - h2) > 1e-12 * hmax) return TB_ERR_NOT_SYMMETRIC;
                    }
                }
        }
        // diagonal of S must be positive
        for (int64_t b = d->brow_ptr[i]; b < d->brow_ptr[i + 1]; ++b)
            if (d->bcol[b] == i)
                for (int a = 0; a < ni; ++a)
                    if (!(d->S_vals[boff[b] + (int64_t)a * ni + a] > 0.0)) return TB_ERR_S_NOT_SPD;
    }
    if (!d->H_vals)
        for (int64_t o = 0; o < N; ++o)
            if (!std::isfinite(d->eps[o])) return TB_ERR_INVALID_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
        cudaGetLastError();
        return TB_ERR_NO_DEVICE;
    }
    // ---- padded host copies ----
    std::vector<double> Sp((size_t)nb * 16, 0.0), Hp;
    if (d->H_vals) Hp.assign((size_t)nb * 16, 0.0);
    std::vector<int> browh(n + 1), bcolh(nb);
    for (int i = 0; i <= n; ++i) browh[i] = (int)d->brow_ptr[i];
    for (int64_t b = 0; b < nb; ++b) bcolh[b] = d->bcol[b];
    for (int i = 0; i < n; ++i) {
        const int ni = d->orb_per_atom[i];
        for (int64_t b = d->brow_ptr[i]; b < d->brow_ptr[i + 1]; ++b) {
            const int j = d->bcol[b], nj = d->orb_per_atom[j];
            for (int a = 0; a < ni; ++a)
                for (int c = 0; c < nj; ++c) {
                    Sp[16 * b + 4 * a + c] = d->S_vals[boff[b] + (int64_t)a * nj + c];
                    if (d->H_vals) Hp[16 * b + 4 * a + c] = d->H_vals[boff[b] + (int64_t)a * nj + c];
                }
            if (j == i)
                for (int a = ni; a < 4; ++a) Sp[16 * b + 5 * a] = 1.0;   // padded slot: S = 1, H = 0
        }
    }
    // identity diagonal blocks of S; TB_UNIT_DIAG=0 keeps the diagonal
    // blocks in the FP32 Chebyshev steps
    const char* ud_env = std::getenv("TB_UNIT_DIAG");
    bool unit_diag = !(ud_env && std::atoi(ud_env) == 0);
    for (int i = 0; i < n && unit_diag; ++i) {
        int ndiag = 0;
        for (int64_t b = d->brow_ptr[i]; b < d->brow_ptr[i + 1]; ++b) {
            if (d->bcol[b] != i) continue;
            ++ndiag;
            for (int q = 0; q < 16; ++q)
                if (Sp[16 * b + q] != (q % 5 == 0 ? 1.0 : 0.0)) unit_diag = false;
        }
        if (ndiag != 1) unit_diag = false;
    }
    std::vector<double> epsp((size_t)4 * n, 0.0);
    std::vector<int32_t> o2p(N);
    for (int i = 0; i < n; ++i)
        for (int a = 0; a < d->orb_per_atom[i]; ++a) {
            o2p[ooff[i] + a] = 4 * i + a;
            if (d->eps) epsp[4 * i + a] = d->eps[ooff[i] + a];
        }
    // ---- device ----
    tb_handle* h = new tb_handle();
    h->n_atoms = n;
    h->n_orb = N;
    h->orb_per_atom.assign(d->orb_per_atom, d->orb_per_atom + n);
    h->brow_h.assign(d->brow_ptr, d->brow_ptr + n + 1);
    h->bcol_h.assign(d->bcol, d->bcol + nb);
    h->boff_h = boff;
    h->btrans_h = btrans;
    h->S_h.assign(d->S_vals, d->S_vals + boff[nb]);
    h->ased = d->H_vals == nullptr;
    h->K = d->K;
    if (h->ased) h->eps_h.assign(d->eps, d->eps + N);
    h->orb2pad_h = o2p;
    h->ds.n_atoms = n;
    h->ds.nb = nb;
    h->ds.npad = 4 * n;
    // systems with s-only atoms keep the diagonal block in the product: on
    // water the changed FP32 rounding of the corrections made more of them
    // fall short of inner_lo_tol (7 % more Chebyshev steps, measured)
    const bool s_only = std::any_of(d->orb_per_atom, d->orb_per_atom + n, [](int32_t o) { return o == 1; });
    h->ds.unit_diag = (unit_diag && !s_only) ? 1 : 0;
    cudaGetDevice(&h->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    auto fail = [&](cudaError_t e) {
        cudaGetLastError();
        tb_destroy(h);
        return e == cudaErrorMemoryAllocation ? TB_ERR_OOM : TB_ERR_CUDA;
    };
    cudaError_t e;
    if ((e = cudaMalloc(&h->ds.brow, sizeof(int) * (n + 1))) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&h->ds.bcol, sizeof(int) * nb)) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&h->ds.S, sizeof(double) * 16 * nb)) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&h->ds.H, sizeof(double) * 16 * nb)) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&h->ds.S32, sizeof(float) * 16 * nb)) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&h->ds.S32lo, sizeof(float) * 16 * nb)) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&h->ds.S32T, sizeof(float) * 16 * nb)) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&h->ds.H32hi, sizeof(float) * 16 * nb)) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&h->ds.H32lo, sizeof(float) * 16 * nb)) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&h->orb2pad, sizeof(int32_t) * N)) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&h->eps_pad, sizeof(double) * 4 * n)) != cudaSuccess) return fail(e);
    if ((e = cudaMallocHost(&h->flags_host, NFLAGS * sizeof(int))) != cudaSuccess) return fail(e);
    if ((e = cudaMallocHost(&h->flags_pool, NPOOL * NFLAGS * sizeof(int))) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&h->atom_orb_off, sizeof(int64_t) * (n + 1))) != cudaSuccess) return fail(e);
    if ((e = cudaMemcpyAsync(h->atom_orb_off, ooff.data(), sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice, st)) != cudaSuccess) return fail(e);
    if ((e = cudaMemcpyAsync(h->ds.brow, browh.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice, st)) != cudaSuccess) return fail(e);
    if ((e = cudaMemcpyAsync(h->ds.bcol, bcolh.data(), sizeof(int) * nb, cudaMemcpyHostToDevice, st)) != cudaSuccess) return fail(e);
    if ((e = cudaMemcpyAsync(h->ds.S, Sp.data(), sizeof(double) * 16 * nb, cudaMemcpyHostToDevice, st)) != cudaSuccess) return fail(e);
    {
        const SpmvGroups g = build_spmv_groups(browh, bcolh, n);
        if (g.G > 0) {
            if ((e = cudaMalloc(&h->ds.grp_ptr, sizeof(int) * g.ptr.size())) != cudaSuccess) return fail(e);
            if ((e = cudaMalloc(&h->ds.grp_cols, sizeof(int) * std::max<size_t>(1, g.cols.size()))) != cudaSuccess) return fail(e);
            if ((e = cudaMalloc(&h->ds.blk_loc, sizeof(int) * nb)) != cudaSuccess) return fail(e);
            if ((e = cudaMemcpyAsync(h->ds.grp_ptr, g.ptr.data(), sizeof(int) * g.ptr.size(), cudaMemcpyHostToDevice, st)) != cudaSuccess) return fail(e);
            if ((e = cudaMemcpyAsync(h->ds.grp_cols, g.cols.data(), sizeof(int) * g.cols.size(), cudaMemcpyHostToDevice, st)) != cudaSuccess) return fail(e);
            if ((e = cudaMemcpyAsync(h->ds.blk_loc, g.loc.data(), sizeof(int) * nb, cudaMemcpyHostToDevice, st)) != cudaSuccess) return fail(e);
            // the host vectors are released at scope exit: wait for the copies
            if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return fail(e);
            h->ds.grpG = g.G;
            h->ds.n_groups = g.n_groups;
            h->ds.max_union = g.max_union;
            h->ds.max_gblocks = g.max_gblocks;
        }
    }

    if ((e = cudaMemcpyAsync(h->orb2pad, o2p.data(), sizeof(int32_t) * N, cudaMemcpyHostToDevice, st)) != cudaSuccess) return fail(e);
    if ((e = cudaMemcpyAsync(h->eps_pad, epsp.data(), sizeof(double) * 4 * n, cudaMemcpyHostToDevice, st)) != cudaSuccess) return fail(e);
    if (d->H_vals) {
        if ((e = cudaMemcpyAsync(h->ds.H, Hp.data(), sizeof(double) * 16 * nb, cudaMemcpyHostToDevice, st)) != cudaSuccess) return fail(e);
    } else {
        launch_ased_build(h->ds, h->eps_pad, d->K, st);
        if ((e = cudaGetLastError()) != cudaSuccess) return fail(e);
    }
    // double-float splits of S and H for the mixed path's FP64-accurate products
    launch_split_f64(h->ds.S, h->ds.S32, h->ds.S32lo, 16 * (long long)nb, st);
    launch_transpose_blocks(h->ds.S32, h->ds.S32T, nb, st);
    if (std::any_of(d->orb_per_atom, d->orb_per_atom + n, [](int32_t o) { return o == 1; })) {
        // exact orbital counts for the Chebyshev step: sp atoms first, then s atoms; compact blocks
        std::vector<unsigned char> no(n);
        std::vector<int> order;
        order.reserve(n);
        for (int i = 0; i < n; ++i) no[i] = (unsigned char)d->orb_per_atom[i];
        for (int i = 0; i < n; ++i)
            if (no[i] == 4) order.push_back(i);
        for (int i = 0; i < n; ++i)
            if (no[i] == 1) order.push_back(i);
        std::vector<int2> bm(nb);
        int64_t tot = 0;   // in float4 units
        for (int i = 0; i < n; ++i)
            for (int64_t b = d->brow_ptr[i]; b < d->brow_ptr[i + 1]; ++b) {
                const int j = d->bcol[b];
                bm[b] = make_int2(j, (int)tot | (no[j] == 1 ? (int)0x80000000u : 0));
                tot += (no[i] == 4 && no[j] == 4) ? 4 : 1;
            }
        if (tot >= ((int64_t)1 << 31)) return fail(cudaErrorMemoryAllocation);
        if ((e = cudaMalloc(&h->ds.norb, n)) != cudaSuccess) return fail(e);
        if ((e = cudaMalloc(&h->ds.row_order, sizeof(int) * n)) != cudaSuccess) return fail(e);
        if ((e = cudaMalloc(&h->ds.bmeta, sizeof(int2) * nb)) != cudaSuccess) return fail(e);
        if ((e = cudaMalloc(&h->ds.S32r, sizeof(float4) * std::max<int64_t>(tot, 1))) != cudaSuccess) return fail(e);
        if ((e = cudaMemcpyAsync(h->ds.norb, no.data(), n, cudaMemcpyHostToDevice, st)) != cudaSuccess) return fail(e);
        if ((e = cudaMemcpyAsync(h->ds.row_order, order.data(), sizeof(int) * n, cudaMemcpyHostToDevice, st)) != cudaSuccess) return fail(e);
        if ((e = cudaMemcpyAsync(h->ds.bmeta, bm.data(), sizeof(int2) * nb, cudaMemcpyHostToDevice, st)) != cudaSuccess) return fail(e);
        h->ds.rag = 1;
        launch_compact_blocks(h->ds, st);
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return fail(e);   // host vectors released at scope exit
    }
    launch_split_f64(h->ds.H, h->ds.H32hi, h->ds.H32lo, 16 * (long long)nb, st);
    if ((e = cudaGetLastError()) != cudaSuccess) return fail(e);
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return fail(e);
    if (noalloc_scratch(h->device, &h->noalloc_base) != TB_OK) return fail(cudaErrorUnknown);
    h->sys_atom_off = {0, (int64_t)n};
    h->sys_orb_off = {0, N};
    *out = h;
    return TB_OK;
}

tb_status tb_create_batch(tb_handle** out, const tb_system_desc* descs, int32_t n_systems, void* stream) {
    if (!out) return TB_ERR_INVALID_ARG;
    *out = nullptr;
    if (!descs || n_systems < 1) return TB_ERR_INVALID_ARG;
    const bool h_given = descs[0].H_vals != nullptr;
    std::vector<int32_t> opa;
    std::vector<int64_t> brow{0};
    std::vector<int32_t> bcol;
    std::vector<double> S, H, eps;
    std::vector<int64_t> aoff{0}, ooff{0};
    for (int q = 0; q < n_systems; ++q) {
        const tb_system_desc& d = descs[q];
        if (d.n_atoms < 1 || !d.orb_per_atom || !d.brow_ptr || !d.bcol || !d.S_vals) return TB_ERR_INVALID_ARG;
        if ((d.H_vals != nullptr) != h_given || d.precision != TB_FP64) return TB_ERR_INVALID_ARG;
        if (!h_given && (!d.eps || !(d.K == descs[0].K))) return TB_ERR_INVALID_ARG;
        const int n = d.n_atoms;
        const int64_t a0 = aoff.back();
        if (a0 + n > (int64_t)1 << 28) return TB_ERR_INVALID_ARG;
        // structure checks needed to size the value arrays; tb_create checks the rest
        if (d.brow_ptr[0] != 0) return TB_ERR_INVALID_ARG;
        int64_t N = 0;
        for (int i = 0; i < n; ++i) {
            if (d.orb_per_atom[i] != 1 && d.orb_per_atom[i] != 4) return TB_ERR_INVALID_ARG;
            if (d.brow_ptr[i + 1] < d.brow_ptr[i]) return TB_ERR_INVALID_ARG;
            N += d.orb_per_atom[i];
        }
        int64_t nval = 0;
        for (int i = 0; i < n; ++i)
            for (int64_t b = d.brow_ptr[i]; b < d.brow_ptr[i + 1]; ++b) {
                const int j = d.bcol[b];
                if (j < 0 || j >= n) return TB_ERR_INVALID_ARG;
                nval += (int64_t)d.orb_per_atom[i] * d.orb_per_atom[j];
            }
        opa.insert(opa.end(), d.orb_per_atom, d.orb_per_atom + n);
        const int64_t b0 = brow.back();
        for (int i = 1; i <= n; ++i) brow.push_back(b0 + d.brow_ptr[i]);
        for (int64_t b = 0; b < d.brow_ptr[n]; ++b) bcol.push_back((int32_t)(a0 + d.bcol[b]));
        S.insert(S.end(), d.S_vals, d.S_vals + nval);
        if (h_given) H.insert(H.end(), d.H_vals, d.H_vals + nval);
        else eps.insert(eps.end(), d.eps, d.eps + N);
        aoff.push_back(a0 + n);
        ooff.push_back(ooff.back() + N);
    }
    tb_system_desc m{};
    m.n_atoms = (int32_t)aoff.back();
    m.orb_per_atom = opa.data();
    m.brow_ptr = brow.data();
    m.bcol = bcol.data();
    m.S_vals = S.data();
    m.H_vals = h_given ? H.data() : nullptr;
    m.eps = h_given ? nullptr : eps.data();
    m.K = descs[0].K;
    m.precision = TB_FP64;
    const tb_status s = tb_create(out, &m, stream);
    if (s != TB_OK) return s;
    tb_handle* h = *out;
    h->sys_atom_off = aoff;
    h->sys_orb_off = ooff;
    if (n_systems == 1) return TB_OK;
    // per-system views: local block columns and padded slots
    std::vector<int32_t> bl(bcol.size());
    for (int q = 0; q < n_systems; ++q)
        for (int64_t b = brow[aoff[q]]; b < brow[aoff[q + 1]]; ++b) bl[b] = bcol[b] - (int32_t)aoff[q];
    h->orb2pad_local_h.resize(ooff.back());
    for (int q = 0; q < n_systems; ++q)
        for (int64_t o = ooff[q]; o < ooff[q + 1]; ++o)
            h->orb2pad_local_h[o] = h->orb2pad_h[o] - 4 * (int32_t)aoff[q];
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    auto fail = [&](cudaError_t e) {
        cudaGetLastError();
        tb_destroy(h);
        *out = nullptr;
        return e == cudaErrorMemoryAllocation ? TB_ERR_OOM : TB_ERR_CUDA;
    };
    cudaError_t e;
    if ((e = cudaMalloc(&h->bcol_local, sizeof(int32_t) * bl.size())) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&h->orb2pad_local, sizeof(int32_t) * ooff.back())) != cudaSuccess) return fail(e);
    if ((e = cudaMemcpyAsync(h->bcol_local, bl.data(), sizeof(int32_t) * bl.size(), cudaMemcpyHostToDevice, st)) != cudaSuccess) return fail(e);
    if ((e = cudaMemcpyAsync(h->orb2pad_local, h->orb2pad_local_h.data(), sizeof(int32_t) * ooff.back(),
                             cudaMemcpyHostToDevice, st)) != cudaSuccess) return fail(e);
    if (h->ds.rag) {
        // block metadata with block columns local to their system (the
        // views' indices); the whole handle, whose indices are global,
        // keeps the padded form of the Chebyshev step
        std::vector<int2> bm(bcol.size());
        if ((e = cudaMemcpyAsync(bm.data(), h->ds.bmeta, sizeof(int2) * bm.size(), cudaMemcpyDeviceToHost, st)) != cudaSuccess) return fail(e);
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return fail(e);
        for (size_t b = 0; b < bm.size(); ++b) bm[b].x = bl[b];
        if ((e = cudaMemcpyAsync(h->ds.bmeta, bm.data(), sizeof(int2) * bm.size(), cudaMemcpyHostToDevice, st)) != cudaSuccess) return fail(e);
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return fail(e);
        // per system, its own block-row order in local atom indices
        std::vector<int> lo(aoff.back());
        for (int q = 0; q < n_systems; ++q) {
            int k = (int)aoff[q];
            for (int64_t i = aoff[q]; i < aoff[q + 1]; ++i)
                if (opa[i] == 4) lo[k++] = (int)(i - aoff[q]);
            for (int64_t i = aoff[q]; i < aoff[q + 1]; ++i)
                if (opa[i] == 1) lo[k++] = (int)(i - aoff[q]);
        }
        if ((e = cudaMalloc(&h->row_order_local, sizeof(int) * lo.size())) != cudaSuccess) return fail(e);
        if ((e = cudaMemcpyAsync(h->row_order_local, lo.data(), sizeof(int) * lo.size(), cudaMemcpyHostToDevice, st)) != cudaSuccess) return fail(e);
    }
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return fail(e);
    for (int q = 0; q < n_systems; ++q) {
        DevSystem v = h->ds;
        if (h->ds.rag) {
            v.norb = h->ds.norb + aoff[q];
            v.row_order = h->row_order_local + aoff[q];
        }
        v.n_atoms = (int)(aoff[q + 1] - aoff[q]);
        v.npad = 4 * v.n_atoms;
        v.nb = brow[aoff[q + 1]] - brow[aoff[q]];
        v.brow = h->ds.brow + aoff[q];
        v.bcol = h->bcol_local;
        v.grpG = 0;                 // the grouped SpMV's atom groups are built for the whole handle
        h->sys_ds.push_back(v);
    }
    h->ds.rag = 0;
    return TB_OK;
}

tb_status tb_overlap_bounds_desc(const tb_system_desc* d, double* lo, double* hi) {
    if (!d || !lo || !hi || d->n_atoms < 1 || !d->orb_per_atom || !d->brow_ptr || !d->bcol || !d->S_vals)
        return TB_ERR_INVALID_ARG;
    const int n = d->n_atoms;
    if (d->brow_ptr[0] != 0) return TB_ERR_INVALID_ARG;
    for (int i = 0; i < n; ++i) {
        if (d->orb_per_atom[i] != 1 && d->orb_per_atom[i] != 4) return TB_ERR_INVALID_ARG;
        if (d->brow_ptr[i + 1] < d->brow_ptr[i]) return TB_ERR_INVALID_ARG;
    }
    const int64_t nb = d->brow_ptr[n];
    std::vector<int64_t> boff(nb + 1, 0);
    for (int i = 0; i < n; ++i)
        for (int64_t b = d->brow_ptr[i]; b < d->brow_ptr[i + 1]; ++b) {
            const int j = d->bcol[b];
            if (j < 0 || j >= n) return TB_ERR_INVALID_ARG;
            boff[b + 1] = boff[b] + (int64_t)d->orb_per_atom[i] * d->orb_per_atom[j];
        }
    return lanczos_bounds(n, d->orb_per_atom, d->brow_ptr, d->bcol, boff.data(), d->S_vals, *lo, *hi);
}

tb_status tb_chebyshev_plan(double lo, double hi, double lo_tol, double inner_tol, int32_t cap, int32_t* n,
                            int32_t* n_last, int32_t* rounds, double* gamma, float* omega, int32_t omega_len) {
    if (!n || !n_last || !rounds || !gamma || !(lo_tol > 0.0 && lo_tol < 1.0) || !(inner_tol > 0.0) || cap < 1)
        return TB_ERR_INVALID_ARG;
    const ChebPlan cp = cheb_plan(lo, hi, lo_tol, inner_tol, cap);
    *n = cp.n;
    *n_last = cp.n_last;
    *rounds = cp.R;
    *gamma = cp.gamma;
    if (omega)
        for (int k = 0; k < omega_len; ++k) omega[k] = k < cp.n ? cp.omega[k] : 0.f;
    return TB_OK;
}

tb_status tb_overlap_bounds(tb_handle* h, double* lo, double* hi) {
    if (!h || !lo || !hi) return TB_ERR_INVALID_ARG;
    return s_bounds(h, *lo, *hi);
}

int32_t tb_num_systems(const tb_handle* h) { return h ? (int32_t)h->sys_atom_off.size() - 1 : 0; }

tb_status tb_batch_offsets(const tb_handle* h, int64_t* atom_off, int64_t* orb_off) {
    if (!h) return TB_ERR_INVALID_ARG;
    if (atom_off) std::memcpy(atom_off, h->sys_atom_off.data(), sizeof(int64_t) * h->sys_atom_off.size());
    if (orb_off) std::memcpy(orb_off, h->sys_orb_off.data(), sizeof(int64_t) * h->sys_orb_off.size());
    return TB_OK;
}

tb_status tb_autotune(tb_handle* h, int32_t K, const double* z, const double* w, double g_s,
                      const tb_solve_opts* opts, int32_t iters, tb_tune* out, int32_t max_out, int32_t* n_out,
                      void* stream) {
    if (!h || !w || !out || max_out < 1 || iters < 1 || !std::isfinite(g_s)) return TB_ERR_INVALID_ARG;
    tb_status s;
    if ((s = check_opts(opts)) != TB_OK) return s;
    if ((s = check_shifts(K, z, opts)) != TB_OK) return s;
    for (int k = 0; k < 2 * K; ++k)
        if (!std::isfinite(w[k])) return TB_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int64_t N = h->n_orb;
    const bool cheb = opts->precision == TB_MIXED && opts->inner_method == TB_INNER_CHEBYSHEV;
    std::vector<tb_tune> cand;
    for (int P : {32, 64, 128, 256}) {
        if (P > next_pow2((int)std::min<int64_t>(N, 1 << 30)) && P > 32) continue;
        for (int nw : {2, 4})
            for (int cpt : {4, 2}) {
                if (!cheb && cpt == 2) continue;
                tb_tune t;
                t.panel = P;
                t.streams = nw;
                t.cheb_cpt = cheb ? cpt : 0;
                t.ctas_per_sm = cheb ? (cpt == 4 ? 3 : 4) : 0;
                t.rate = 0.0;
                cand.push_back(t);
            }
    }
    Cleanup cl;
    cl.st = st;
    double* qd = nullptr;
    const int Rmax = (int)std::min<int64_t>(N, 4 * 256);
    if ((s = dalloc(cl, &qd, (size_t)Rmax)) != TB_OK) return s;
    cudaEvent_t e0, e1;
    TB_CK(cudaEventCreate(&e0));
    TB_CK(cudaEventCreate(&e1));
    for (auto& t : cand) {
        // as many panels as are kept in flight, columns spread over the system
        const int R = (int)std::min<int64_t>(N, (int64_t)t.panel * t.streams);
        std::vector<int32_t> cols(R);
        for (int c = 0; c < R; ++c) cols[c] = (int32_t)(((int64_t)c * N) / R);
        tb_solve_opts oc = *opts;
        oc.panel = t.panel;
        oc.max_iter = iters;
        Solve q;
        q.K = K; q.z = z; q.R = R; q.cols = cols.data(); q.proj = PROJ_SROW; q.w = w; q.g_s = g_s; q.q_out = qd;
        q.streams = t.streams;
        q.cheb_cpt = t.cheb_cpt;
        // the first call builds the graphs and the spectrum bounds; the second is timed
        tb_status r = run_solve(h, q, &oc, nullptr, st);
        if (r != TB_OK && r != TB_ERR_NOT_CONVERGED) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return r;
        }
        TB_CK(cudaEventRecord(e0, st));
        r = run_solve(h, q, &oc, nullptr, st);
        TB_CK(cudaEventRecord(e1, st));
        TB_CK(cudaEventSynchronize(e1));
        float ms = 0.f;
        TB_CK(cudaEventElapsedTime(&ms, e0, e1));
        if (r != TB_OK && r != TB_ERR_NOT_CONVERGED) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return r;
        }
        t.rate = ms > 0.f ? (double)K * R * iters / (ms * 1e-3) : 0.0;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    std::stable_sort(cand.begin(), cand.end(), [](const tb_tune& a, const tb_tune& b) { return a.rate > b.rate; });
    const tb_tune& best = cand.front();
    {
        std::lock_guard<std::mutex> lk(h->tune_mu);
        const int kb = next_pow2(K);
        tb_handle::Tuned t{opts->precision, opts->inner_method, kb, best.panel, best.streams, best.cheb_cpt, best.rate};
        bool found = false;
        for (auto& x : h->tuned)
            if (x.prec == t.prec && x.method == t.method && x.kb == t.kb) {
                x = t;
                found = true;
            }
        if (!found) h->tuned.push_back(t);
    }
    const int n = std::min<int>(max_out, (int)cand.size());
    for (int i = 0; i < n; ++i) out[i] = cand[i];
    if (n_out) *n_out = n;
    return TB_OK;
}

tb_status tb_shifted_cocg(tb_handle* h, int32_t K, const double* z, int32_t R, const int32_t* cols,
                          const tb_solve_opts* opts, double* x_out, tb_stats* stats, void* stream) {
    if (!h || !x_out) return TB_ERR_INVALID_ARG;
    tb_status s;
    if ((s = check_opts(opts)) != TB_OK) return s;
    if ((s = check_shifts(K, z, opts)) != TB_OK) return s;
    if ((s = check_cols(h, R, cols)) != TB_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // energy-point checkpointing: shifts per chunk so that x^k, p^k of the
    // panels in flight and the device copy of the chunk's solutions fit the
    // state budget (x_out is [K][R][N]: a chunk of shifts is one contiguous
    // slice of it)
    const int64_t N = h->n_orb;
    const bool host_out = !is_device_ptr(x_out);
    const int Pw = std::min(opts->panel ? opts->panel : 64, next_pow2(R));
    const int inflight = std::min<int64_t>(workers_for(h), (R + Pw - 1) / Pw);
    const double per_shift = 32.0 * (double)h->ds.npad * Pw * inflight + (host_out ? 16.0 * (double)R * N : 0.0);
    const int Kc = (int)std::max<double>(1.0, std::min<double>(K, std::floor((double)state_budget(opts) / per_shift)));
    Cleanup cl;
    cl.st = st;
    OutBuf ob;
    if ((s = out_prepare(cl, ob, x_out, sizeof(double2) * (size_t)Kc * R * N)) != TB_OK) return s;
    const auto t0 = std::chrono::steady_clock::now();
    tb_stats agg{};
    std::vector<int32_t> conv;
    bool unconverged = false;
    for (int k0 = 0; k0 < K; k0 += Kc) {
        const int kc = std::min(Kc, K - k0);
        const tb_solve_opts oc = chunk_opts(opts, k0, kc);
        Solve q;
        q.K = kc; q.z = z + 2 * (size_t)k0; q.R = R; q.cols = cols; q.proj = PROJ_NONE;
        q.x_out = ob.host ? static_cast<double2*>(ob.dev) : reinterpret_cast<double2*>(x_out) + (size_t)k0 * R * N;
        tb_stats ts{};
        if (stats && stats->conv_iter) {
            conv.assign((size_t)R * kc, -1);
            ts.conv_iter = conv.data();
        }
        const tb_status run = run_solve(h, q, &oc, stats ? &ts : nullptr, st);
        if (run == TB_ERR_NOT_CONVERGED) unconverged = true;
        else if (run != TB_OK) return run;
        if (ob.host) {
            // the chunk's solutions to the caller's host memory before the next chunk reuses the device copy
            TB_CK(cudaMemcpyAsync(reinterpret_cast<double2*>(x_out) + (size_t)k0 * R * N, ob.dev,
                                  sizeof(double2) * (size_t)kc * R * N, cudaMemcpyDeviceToHost, st));
        }
        TB_CK(cudaStreamSynchronize(st));
        if (stats) {
            if (stats->conv_iter)
                for (int c = 0; c < R; ++c)
                    for (int k = 0; k < kc; ++k) stats->conv_iter[(size_t)c * K + k0 + k] = conv[(size_t)c * kc + k];
            agg.outer_iterations += ts.outer_iterations;
            agg.inner_iterations += ts.inner_iterations;
            agg.max_column_iterations = std::max(agg.max_column_iterations, ts.max_column_iterations);
            agg.switches += ts.switches;
            agg.unconverged += ts.unconverged;
            agg.inner_redos += ts.inner_redos;
        }
    }
    if (stats) {
        int32_t* ci = stats->conv_iter;
        *stats = agg;
        stats->conv_iter = ci;
        stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    return unconverged ? TB_ERR_NOT_CONVERGED : TB_OK;
}

tb_status tb_green_elements(tb_handle* h, int32_t K, const double* z, int32_t R, const int32_t* cols,
                            const int64_t* row_ptr, const int32_t* rows, const tb_solve_opts* opts,
                            double* G_out, tb_stats* stats, void* stream) {
    return tb_green_elements_dz(h, K, z, R, cols, row_ptr, rows, opts, G_out, nullptr, stats, stream);
}

tb_status tb_green_elements_dz(tb_handle* h, int32_t K, const double* z, int32_t R, const int32_t* cols,
                               const int64_t* row_ptr, const int32_t* rows, const tb_solve_opts* opts,
                               double* G_out, double* dG_out, tb_stats* stats, void* stream) {
    if (!h || !G_out || !row_ptr || !rows) return TB_ERR_INVALID_ARG;
    tb_status s;
    if ((s = check_opts(opts)) != TB_OK) return s;
    if ((s = check_shifts(K, z, opts)) != TB_OK) return s;
    if ((s = check_cols(h, R, cols)) != TB_OK) return s;
    if (row_ptr[0] != 0) return TB_ERR_INVALID_ARG;
    for (int c = 0; c < R; ++c) {
        const int64_t m = row_ptr[c + 1] - row_ptr[c];
        if (m < 1 || m > MAX_M) return TB_ERR_INVALID_ARG;
    }
    for (int64_t e = 0; e < row_ptr[R]; ++e)
        if (rows[e] < 0 || rows[e] >= h->n_orb) return TB_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Cleanup cl;
    cl.st = st;
    OutBuf ob, obd;
    const size_t bytes = sizeof(double2) * (size_t)row_ptr[R] * K;
    if ((s = out_prepare(cl, ob, G_out, bytes)) != TB_OK) return s;
    if (dG_out && (s = out_prepare(cl, obd, dG_out, bytes)) != TB_OK) return s;
    Solve q;
    q.K = K; q.z = z; q.R = R; q.cols = cols; q.proj = PROJ_ROWS; q.row_ptr = row_ptr; q.rows = rows;
    q.g_out = static_cast<double2*>(ob.dev);
    q.dg_out = dG_out ? static_cast<double2*>(obd.dev) : nullptr;
    const tb_status run = run_solve(h, q, opts, stats, st);
    tb_status fin = out_finish(ob, st);
    if (dG_out && fin == TB_OK) fin = out_finish(obd, st);
    return merge(run, fin);
}

tb_status tb_forces(tb_handle* h, const double* dE_dH, const double* dE_dS, const double* dS_dd, const double* dH_dd,
                    double* F_out, void* stream) {
    if (!h || !dE_dH || !dE_dS || !dS_dd || !F_out) return TB_ERR_INVALID_ARG;
    if (!dH_dd && !h->ased) return TB_ERR_INVALID_ARG;   // no rule for dH/dd of an explicit H
    const int n = h->n_atoms;
    const int64_t nb = (int64_t)h->bcol_h.size();
    const int64_t nvals = h->boff_h.back();
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Cleanup cl;
    cl.st = st;
    tb_status s;
    const double *gH, *gS, *dS, *dH = nullptr, *eps = nullptr;
    if ((s = device_view(cl, dE_dH, (size_t)nvals, &gH, st)) != TB_OK) return s;
    if ((s = device_view(cl, dE_dS, (size_t)nvals, &gS, st)) != TB_OK) return s;
    if ((s = device_view(cl, dS_dd, (size_t)3 * nvals, &dS, st)) != TB_OK) return s;
    if (dH_dd && (s = device_view(cl, dH_dd, (size_t)3 * nvals, &dH, st)) != TB_OK) return s;
    if (!dH_dd && (s = device_view(cl, h->eps_h.data(), h->eps_h.size(), &eps, st)) != TB_OK) return s;
    const int64_t *boff, *btr;
    if ((s = device_view(cl, h->boff_h.data(), h->boff_h.size(), &boff, st)) != TB_OK) return s;
    if ((s = device_view(cl, h->btrans_h.data(), h->btrans_h.size(), &btr, st)) != TB_OK) return s;
    double* vblk = nullptr;
    if ((s = dalloc(cl, &vblk, (size_t)3 * nb)) != TB_OK) return s;
    OutBuf ob;
    if ((s = out_prepare(cl, ob, F_out, sizeof(double) * 3 * (size_t)n)) != TB_OK) return s;
    launch_force_blocks(n, h->ds.brow, h->ds.bcol, boff, h->atom_orb_off, gH, gS, dS, dH, eps, h->K, nvals, vblk, st);
    launch_force_atoms(n, h->ds.brow, h->ds.bcol, btr, vblk, static_cast<double*>(ob.dev), st);
    TB_CK(cudaGetLastError());
    return out_finish(ob, st);
}

tb_status tb_mulliken_vjp(tb_handle* h, int32_t K, const double* z, const double* w, double g_s, const double* v,
                          const tb_solve_opts* opts, double* dL_dH, double* dL_dS, tb_stats* stats, void* stream) {
    if (!h || !w || !v || !dL_dH || !dL_dS || !std::isfinite(g_s)) return TB_ERR_INVALID_ARG;
    if (h->sys_atom_off.size() > 2) return TB_ERR_INVALID_ARG;   // one system per handle
    tb_status s;
    if ((s = check_opts(opts)) != TB_OK) return s;
    if ((s = check_shifts(K, z, opts)) != TB_OK) return s;
    for (int k = 0; k < 2 * K; ++k)
        if (!std::isfinite(w[k])) return TB_ERR_INVALID_ARG;
    const auto t0 = std::chrono::steady_clock::now();
    const int n = h->n_atoms;
    const int64_t N = h->n_orb;
    const int64_t nvals = h->boff_h.back();
    std::vector<int64_t> ooff(n + 1, 0);
    for (int i = 0; i < n; ++i) ooff[i + 1] = ooff[i] + h->orb_per_atom[i];
    // every stored entry (a, b) in the caller's block layout
    std::vector<int32_t> ea(nvals), eb(nvals);
    for (int I = 0; I < n; ++I)
        for (int64_t blk = h->brow_h[I]; blk < h->brow_h[I + 1]; ++blk) {
            const int J = h->bcol_h[blk];
            const int ni = h->orb_per_atom[I], nj = h->orb_per_atom[J];
            for (int ai = 0; ai < ni; ++ai)
                for (int bj = 0; bj < nj; ++bj) {
                    const int64_t e = h->boff_h[blk] + (int64_t)ai * nj + bj;
                    ea[e] = (int32_t)(ooff[I] + ai);
                    eb[e] = (int32_t)(ooff[J] + bj);
                }
        }
    // the columns c with v_c != 0: only they enter G S D_v G and v_b G_ba
    std::vector<double> vh((size_t)N);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (is_device_ptr(v)) {
        TB_CK(cudaMemcpyAsync(vh.data(), v, sizeof(double) * N, cudaMemcpyDeviceToHost, st));
        TB_CK(cudaStreamSynchronize(st));
    } else {
        std::memcpy(vh.data(), v, sizeof(double) * N);
    }
    std::vector<int32_t> supp;
    for (int64_t o = 0; o < N; ++o) {
        if (!std::isfinite(vh[o])) return TB_ERR_INVALID_ARG;
        if (vh[o] != 0.0) supp.push_back((int32_t)o);
    }
    const int64_t ns = (int64_t)supp.size();
    // columns and shifts per chunk (energy-point checkpointing): the two
    // full-solution panels X, Y ([Kc][Rc][N]) and the solver's x^k, p^k of
    // the same shifts and columns, ~64 N bytes per (column, shift), within
    // the state budget; all K shifts at once while one column fits, else
    // chunks of shifts, each solved again from its own seed sequence
    const double per_cs = 64.0 * (double)N;
    const double budget = (double)state_budget(opts);
    const int Rc = (int)std::max<double>(1.0, std::min<double>(std::max<int64_t>(ns, 1), std::floor(budget / (per_cs * K))));
    const int Kc = (int)std::max<double>(1.0, std::min<double>(K, std::floor(budget / (per_cs * Rc))));
    Cleanup cl;
    cl.st = st;
    int32_t *ead, *ebd, *cpos;
    double *gH, *gS, *Sc, *vc;
    double2 *X, *Y, *zd, *wd;
    if ((s = dalloc(cl, &cpos, (size_t)N)) != TB_OK) return s;
    if ((s = dalloc(cl, &vc, (size_t)Rc)) != TB_OK) return s;
    if ((s = dalloc(cl, &ead, (size_t)nvals)) != TB_OK) return s;
    if ((s = dalloc(cl, &ebd, (size_t)nvals)) != TB_OK) return s;
    if ((s = dalloc(cl, &gH, (size_t)nvals)) != TB_OK) return s;
    if ((s = dalloc(cl, &gS, (size_t)nvals)) != TB_OK) return s;
    if ((s = dalloc(cl, &Sc, (size_t)Rc * N)) != TB_OK) return s;
    if ((s = dalloc(cl, &X, (size_t)Kc * Rc * N)) != TB_OK) return s;
    if ((s = dalloc(cl, &Y, (size_t)Kc * Rc * N)) != TB_OK) return s;
    if ((s = dalloc(cl, &zd, (size_t)K)) != TB_OK) return s;
    if ((s = dalloc(cl, &wd, (size_t)K)) != TB_OK) return s;
    TB_CK(cudaMemcpyAsync(ead, ea.data(), sizeof(int32_t) * nvals, cudaMemcpyHostToDevice, st));
    TB_CK(cudaMemcpyAsync(ebd, eb.data(), sizeof(int32_t) * nvals, cudaMemcpyHostToDevice, st));
    TB_CK(cudaMemcpyAsync(zd, z, sizeof(double2) * K, cudaMemcpyHostToDevice, st));
    TB_CK(cudaMemcpyAsync(wd, w, sizeof(double2) * K, cudaMemcpyHostToDevice, st));
    TB_CK(cudaMemsetAsync(gH, 0, sizeof(double) * nvals, st));
    TB_CK(cudaMemsetAsync(gS, 0, sizeof(double) * nvals, st));
    View vw = whole_view(h);
    tb_stats agg{};
    bool unconverged = false;
    std::vector<double> Sh((size_t)Rc * N);
    std::vector<int32_t> cols(Rc), cposh((size_t)N, -1);
    std::vector<double> vch(Rc);
    for (int64_t c0 = 0; c0 < ns; c0 += Rc) {
        const int rc = (int)std::min<int64_t>(Rc, ns - c0);
        // columns s_c of S (= rows, S symmetric) in caller order; the
        // chunk position of every orbital that is one of its columns
        std::fill(Sh.begin(), Sh.end(), 0.0);
        if (c0 > 0)
            for (int64_t q = c0 - Rc; q < c0; ++q) cposh[supp[q]] = -1;
        for (int c = 0; c < rc; ++c) {
            const int64_t o = supp[c0 + c];
            cols[c] = (int32_t)o;
            cposh[o] = c;
            vch[c] = vh[o];
            const int J = (int)(std::upper_bound(ooff.begin(), ooff.end(), o) - ooff.begin()) - 1;
            const int bj = (int)(o - ooff[J]);
            for (int64_t blk = h->brow_h[J]; blk < h->brow_h[J + 1]; ++blk) {
                const int I = h->bcol_h[blk];
                const int ni = h->orb_per_atom[I];
                for (int ai = 0; ai < ni; ++ai)
                    Sh[(size_t)c * N + ooff[I] + ai] = h->S_h[h->boff_h[blk] + (int64_t)bj * ni + ai];
            }
        }
        TB_CK(cudaMemcpyAsync(Sc, Sh.data(), sizeof(double) * (size_t)rc * N, cudaMemcpyHostToDevice, st));
        TB_CK(cudaMemcpyAsync(cpos, cposh.data(), sizeof(int32_t) * N, cudaMemcpyHostToDevice, st));
        TB_CK(cudaMemcpyAsync(vc, vch.data(), sizeof(double) * rc, cudaMemcpyHostToDevice, st));
        for (int k0 = 0; k0 < K; k0 += Kc) {
            const int kc = std::min(Kc, K - k0);
            const tb_solve_opts oc = chunk_opts(opts, k0, kc);
            for (int pass = 0; pass < 2; ++pass) {
                Solve q;
                q.K = kc; q.z = z + 2 * (size_t)k0; q.R = rc; q.cols = cols.data(); q.proj = PROJ_NONE;
                q.x_out = pass == 0 ? X : Y;
                if (pass == 1) q.rhs = Sc;
                tb_stats ts{};
                const tb_status run = run_view(vw, q, &oc, &ts, st);
                if (run == TB_ERR_NOT_CONVERGED) unconverged = true;
                else if (run != TB_OK) return run;
                agg.outer_iterations += ts.outer_iterations;
                agg.inner_iterations += ts.inner_iterations;
                agg.max_column_iterations = std::max(agg.max_column_iterations, ts.max_column_iterations);
                agg.switches += ts.switches;
                agg.unconverged += ts.unconverged;
                agg.inner_redos += ts.inner_redos;
            }
            // this chunk's shifts add their terms of the k sums
            launch_vjp_accumulate(X, Y, kc, rc, N, cpos, vc, ead, ebd, nvals, zd + k0, wd + k0, g_s, gH, gS, st);
            TB_CK(cudaGetLastError());
        }
        TB_CK(cudaStreamSynchronize(st));   // the host staging arrays are refilled for the next chunk
    }
    OutBuf oH, oS;
    if ((s = out_prepare(cl, oH, dL_dH, sizeof(double) * nvals)) != TB_OK) return s;
    if ((s = out_prepare(cl, oS, dL_dS, sizeof(double) * nvals)) != TB_OK) return s;
    TB_CK(cudaMemcpyAsync(oH.dev, gH, sizeof(double) * nvals, cudaMemcpyDeviceToDevice, st));
    TB_CK(cudaMemcpyAsync(oS.dev, gS, sizeof(double) * nvals, cudaMemcpyDeviceToDevice, st));
    tb_status fin = out_finish(oH, st);
    if (fin == TB_OK) fin = out_finish(oS, st);
    if (stats) {
        int32_t* ci = stats->conv_iter;
        *stats = agg;
        stats->conv_iter = ci;
        stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    if (fin != TB_OK) return fin;
    return unconverged ? TB_ERR_NOT_CONVERGED : TB_OK;
}

// Every column b of the H/S pattern with the rows a of its block column, in
// caller orbital order; element e = (a, b) also names the value index
// val[e] of H_ab / S_ab in the caller's block layout, S_el[e] = S_ab, and the
// atoms of a and b.
struct PatternElems {
    std::vector<int32_t> cols, rows, atom_a, atom_b;
    std::vector<int64_t> row_ptr, val;
    std::vector<double> S_el;
};

static tb_status pattern_elements(const tb_handle* h, PatternElems& pe) {
    const int n = h->n_atoms;
    const int64_t N = h->n_orb;
    std::vector<int64_t> ooff(n + 1, 0);
    for (int i = 0; i < n; ++i) ooff[i + 1] = ooff[i] + h->orb_per_atom[i];
    pe.cols.assign(N, 0);
    pe.row_ptr.assign(N + 1, 0);
    for (int J = 0; J < n; ++J) {
        const int nj = h->orb_per_atom[J];
        for (int bo = 0; bo < nj; ++bo) {
            const int64_t b = ooff[J] + bo;
            pe.cols[b] = (int32_t)b;
            // block column J = block row J by symmetry of the pattern
            for (int64_t blk = h->brow_h[J]; blk < h->brow_h[J + 1]; ++blk) {
                const int I = h->bcol_h[blk];
                const int ni = h->orb_per_atom[I];
                const int64_t bt = h->btrans_h[blk];       // block (I, J)
                for (int ao = 0; ao < ni; ++ao) {
                    pe.rows.push_back((int32_t)(ooff[I] + ao));
                    const int64_t v = h->boff_h[bt] + (int64_t)ao * nj + bo;
                    pe.val.push_back(v);
                    pe.S_el.push_back(h->S_h[v]);
                    pe.atom_a.push_back(I);
                    pe.atom_b.push_back(J);
                }
            }
            pe.row_ptr[b + 1] = (int64_t)pe.rows.size();
            if (pe.row_ptr[b + 1] - pe.row_ptr[b] > MAX_M) return TB_ERR_INVALID_ARG;
        }
    }
    return TB_OK;
}

tb_status tb_band_energy(tb_handle* h, int32_t K, const double* z, const double* w, double g_s,
                         const tb_solve_opts* opts, double* E_out, double* dE_dH, double* dE_dS, tb_stats* stats,
                         void* stream) {
    if (!h || !E_out || !dE_dH || !dE_dS || !w || !std::isfinite(g_s)) return TB_ERR_INVALID_ARG;
    tb_status s;
    if ((s = check_opts(opts)) != TB_OK) return s;
    if ((s = check_shifts(K, z, opts)) != TB_OK) return s;
    for (int k = 0; k < 2 * K; ++k)
        if (!std::isfinite(w[k])) return TB_ERR_INVALID_ARG;
    const int64_t N = h->n_orb;
    PatternElems pe;
    if ((s = pattern_elements(h, pe)) != TB_OK) return s;
    const std::vector<int32_t>& cols = pe.cols;
    const std::vector<int32_t>& rows = pe.rows;
    const std::vector<int64_t>& row_ptr = pe.row_ptr;
    const std::vector<int64_t>& val = pe.val;
    const std::vector<double>& S_el = pe.S_el;
    const int64_t ne = (int64_t)rows.size();
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Cleanup cl;
    cl.st = st;
    double2 *G, *dG, *zd, *wd;
    double *Sd, *et, *gH, *gS, *Ed;
    int64_t* vald;
    if ((s = dalloc(cl, &G, (size_t)ne * K)) != TB_OK) return s;
    if ((s = dalloc(cl, &dG, (size_t)ne * K)) != TB_OK) return s;
    if ((s = dalloc(cl, &zd, (size_t)K)) != TB_OK) return s;
    if ((s = dalloc(cl, &wd, (size_t)K)) != TB_OK) return s;
    if ((s = dalloc(cl, &Sd, (size_t)ne)) != TB_OK) return s;
    if ((s = dalloc(cl, &et, (size_t)ne)) != TB_OK) return s;
    if ((s = dalloc(cl, &gH, (size_t)ne)) != TB_OK) return s;
    if ((s = dalloc(cl, &gS, (size_t)ne)) != TB_OK) return s;
    if ((s = dalloc(cl, &Ed, 1)) != TB_OK) return s;
    if ((s = dalloc(cl, &vald, (size_t)ne)) != TB_OK) return s;
    TB_CK(cudaMemcpyAsync(zd, z, sizeof(double2) * K, cudaMemcpyHostToDevice, st));
    TB_CK(cudaMemcpyAsync(wd, w, sizeof(double2) * K, cudaMemcpyHostToDevice, st));
    TB_CK(cudaMemcpyAsync(Sd, S_el.data(), sizeof(double) * ne, cudaMemcpyHostToDevice, st));
    TB_CK(cudaMemcpyAsync(vald, val.data(), sizeof(int64_t) * ne, cudaMemcpyHostToDevice, st));
    Solve q;
    q.K = K; q.z = z; q.R = (int)N; q.cols = cols.data(); q.proj = PROJ_ROWS; q.row_ptr = row_ptr.data();
    q.rows = rows.data(); q.g_out = G; q.dg_out = dG;
    const tb_status run = run_solve(h, q, opts, stats, st);
    if (run != TB_OK && run != TB_ERR_NOT_CONVERGED) return run;
    launch_band_energy_terms(G, dG, Sd, ne, K, zd, wd, g_s, et, gH, gS, st);
    launch_sum_fixed(et, ne, Ed, st);
    // gradients into the caller's block layout (every pattern value once)
    const size_t nval = (size_t)h->boff_h.back();
    OutBuf oH, oS, oE;
    if ((s = out_prepare(cl, oH, dE_dH, sizeof(double) * nval)) != TB_OK) return s;
    if ((s = out_prepare(cl, oS, dE_dS, sizeof(double) * nval)) != TB_OK) return s;
    if ((s = out_prepare(cl, oE, E_out, sizeof(double))) != TB_OK) return s;
    launch_scatter_values(gH, vald, ne, static_cast<double*>(oH.dev), st);
    launch_scatter_values(gS, vald, ne, static_cast<double*>(oS.dev), st);
    TB_CK(cudaMemcpyAsync(oE.dev, Ed, sizeof(double), cudaMemcpyDeviceToDevice, st));
    TB_CK(cudaGetLastError());
    tb_status fin = out_finish(oH, st);
    if (fin == TB_OK) fin = out_finish(oS, st);
    if (fin == TB_OK) fin = out_finish(oE, st);
    return merge(run, fin);
}

tb_status tb_mulliken_orbital(tb_handle* h, int32_t K, const double* z, const double* w, double g_s,
                              int32_t R, const int32_t* cols, const tb_solve_opts* opts, double* q_out,
                              tb_stats* stats, void* stream) {
    if (!h || !q_out || !w || !std::isfinite(g_s)) return TB_ERR_INVALID_ARG;
    tb_status s;
    if ((s = check_opts(opts)) != TB_OK) return s;
    if ((s = check_shifts(K, z, opts)) != TB_OK) return s;
    if ((s = check_cols(h, R, cols)) != TB_OK) return s;
    for (int k = 0; k < 2 * K; ++k)
        if (!std::isfinite(w[k])) return TB_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Cleanup cl;
    cl.st = st;
    OutBuf ob;
    if ((s = out_prepare(cl, ob, q_out, sizeof(double) * (size_t)R)) != TB_OK) return s;
    Solve q;
    q.K = K; q.z = z; q.R = R; q.cols = cols; q.proj = PROJ_SROW; q.w = w; q.g_s = g_s;
    q.q_out = static_cast<double*>(ob.dev);
    const tb_status run = run_solve(h, q, opts, stats, st);
    return merge(run, out_finish(ob, st));
}


tb_status tb_mulliken_charges(tb_handle* h, int32_t K, const double* z, const double* w, double g_s,
                              const tb_solve_opts* opts, double* q_out, tb_stats* stats, void* stream) {
    if (!h || !q_out) return TB_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Cleanup cl;
    cl.st = st;
    OutBuf ob;
    tb_status s;
    if ((s = out_prepare(cl, ob, q_out, sizeof(double) * (size_t)h->n_atoms)) != TB_OK) return s;
    const tb_status run = mulliken_atoms_device(h, K, z, w, g_s, opts, static_cast<double*>(ob.dev), stats, st);
    if (run != TB_OK && run != TB_ERR_NOT_CONVERGED) return run;
    return merge(run, out_finish(ob, st));
}

// ---- charge self-consistency (Eq. Hap-CSC) ---------------------------------

void tb_default_csc_opts(tb_csc_opts* o) {
    if (!o) return;
    o->max_scf = 50;
    o->scf_tol = 1e-6;
    o->mix = 0.3;
}


tb_status tb_csc_hamiltonian(tb_handle* h, const double* gamma, const double* dq, void* stream) {
    if (!h) return TB_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (!dq) {
        if (h->H0) {
            TB_CK(cudaMemcpyAsync(h->ds.H, h->H0, sizeof(double) * 16 * (size_t)h->ds.nb, cudaMemcpyDeviceToDevice, st));
            launch_split_f64(h->ds.H, h->ds.H32hi, h->ds.H32lo, 16 * (long long)h->ds.nb, st);
            TB_CK(cudaGetLastError());
        }
        TB_CK(cudaStreamSynchronize(st));
        return TB_OK;
    }
    if (!gamma) return TB_ERR_INVALID_ARG;
    tb_status s;
    if ((s = ensure_H0(h, st)) != TB_OK) return s;
    Cleanup cl;
    cl.st = st;
    const int n = h->n_atoms;
    const double *gd = nullptr, *dqd = nullptr;
    double* V = nullptr;
    if ((s = device_view(cl, gamma, (size_t)n * n, &gd, st)) != TB_OK) return s;
    if ((s = device_view(cl, dq, (size_t)n, &dqd, st)) != TB_OK) return s;
    if ((s = dalloc(cl, &V, (size_t)n)) != TB_OK) return s;
    launch_csc_potential(gd, dqd, n, V, st);
    launch_csc_hamiltonian(h->ds, h->H0, V, st);
    TB_CK(cudaGetLastError());
    TB_CK(cudaStreamSynchronize(st));
    return TB_OK;
}

tb_status tb_csc_forces(tb_handle* h, int32_t K, const double* z, const double* w, double g_s, const double* gamma,
                        const double* dgamma, const double* dq, const double* dS_dd, const tb_solve_opts* opts,
                        double* F_out, tb_stats* stats, void* stream) {
    if (!h || !w || !gamma || !dgamma || !dq || !dS_dd || !F_out || !std::isfinite(g_s)) return TB_ERR_INVALID_ARG;
    if (!h->ased) return TB_ERR_INVALID_ARG;                       // dH0/dR by Eq. Hap-1 needs eps and K
    if (h->sys_atom_off.size() > 2) return TB_ERR_INVALID_ARG;     // one system per handle
    tb_status s;
    if ((s = check_opts(opts)) != TB_OK) return s;
    if ((s = check_shifts(K, z, opts)) != TB_OK) return s;
    for (int k = 0; k < 2 * K; ++k)
        if (!std::isfinite(w[k])) return TB_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int n = h->n_atoms;
    // H = H0 + H^CSC(dq) on the handle (left there, as tb_csc_hamiltonian)
    if ((s = tb_csc_hamiltonian(h, gamma, dq, stream)) != TB_OK) return s;
    PatternElems pe;
    if ((s = pattern_elements(h, pe)) != TB_OK) return s;
    const int64_t ne = (int64_t)pe.rows.size();
    const int64_t nvals = h->boff_h.back();
    Cleanup cl;
    cl.st = st;
    const double *gd = nullptr, *dqd = nullptr, *dgd = nullptr;
    if ((s = device_view(cl, gamma, (size_t)n * n, &gd, st)) != TB_OK) return s;
    if ((s = device_view(cl, dq, (size_t)n, &dqd, st)) != TB_OK) return s;
    if ((s = device_view(cl, dgamma, (size_t)n * n * 3, &dgd, st)) != TB_OK) return s;
    double2 *G, *zd, *wd;
    double *V, *gHe, *gSe, *gHv, *gSv, *F;
    int32_t *aa, *ab;
    int64_t* vald;
    if ((s = dalloc(cl, &G, (size_t)ne * K)) != TB_OK) return s;
    if ((s = dalloc(cl, &zd, (size_t)K)) != TB_OK) return s;
    if ((s = dalloc(cl, &wd, (size_t)K)) != TB_OK) return s;
    if ((s = dalloc(cl, &V, (size_t)n)) != TB_OK) return s;
    if ((s = dalloc(cl, &gHe, (size_t)ne)) != TB_OK) return s;
    if ((s = dalloc(cl, &gSe, (size_t)ne)) != TB_OK) return s;
    if ((s = dalloc(cl, &gHv, (size_t)nvals)) != TB_OK) return s;
    if ((s = dalloc(cl, &gSv, (size_t)nvals)) != TB_OK) return s;
    if ((s = dalloc(cl, &F, (size_t)3 * n)) != TB_OK) return s;
    if ((s = dalloc(cl, &aa, (size_t)ne)) != TB_OK) return s;
    if ((s = dalloc(cl, &ab, (size_t)ne)) != TB_OK) return s;
    if ((s = dalloc(cl, &vald, (size_t)ne)) != TB_OK) return s;
    TB_CK(cudaMemcpyAsync(zd, z, sizeof(double2) * K, cudaMemcpyHostToDevice, st));
    TB_CK(cudaMemcpyAsync(wd, w, sizeof(double2) * K, cudaMemcpyHostToDevice, st));
    TB_CK(cudaMemcpyAsync(aa, pe.atom_a.data(), sizeof(int32_t) * ne, cudaMemcpyHostToDevice, st));
    TB_CK(cudaMemcpyAsync(ab, pe.atom_b.data(), sizeof(int32_t) * ne, cudaMemcpyHostToDevice, st));
    TB_CK(cudaMemcpyAsync(vald, pe.val.data(), sizeof(int64_t) * ne, cudaMemcpyHostToDevice, st));
    launch_csc_potential(gd, dqd, n, V, st);
    Solve q;
    q.K = K; q.z = z; q.R = (int)h->n_orb; q.cols = pe.cols.data(); q.proj = PROJ_ROWS;
    q.row_ptr = pe.row_ptr.data(); q.rows = pe.rows.data(); q.g_out = G;
    const tb_status run = run_solve(h, q, opts, stats, st);
    if (run != TB_OK && run != TB_ERR_NOT_CONVERGED) return run;
    launch_csc_force_terms(G, ne, K, zd, wd, g_s, V, aa, ab, gHe, gSe, st);
    TB_CK(cudaMemsetAsync(gHv, 0, sizeof(double) * nvals, st));
    TB_CK(cudaMemsetAsync(gSv, 0, sizeof(double) * nvals, st));
    launch_scatter_values(gHe, vald, ne, gHv, st);
    launch_scatter_values(gSe, vald, ne, gSv, st);
    TB_CK(cudaGetLastError());
    // the force blocks of Eq. Hap-1 with gH = rho^T and gS as above, then
    // the Coulomb-gradient term
    if ((s = tb_forces(h, gHv, gSv, dS_dd, nullptr, F, stream)) != TB_OK) return s;
    launch_csc_force_coulomb(n, dgd, dqd, F, st);
    TB_CK(cudaGetLastError());
    OutBuf ob;
    if ((s = out_prepare(cl, ob, F_out, sizeof(double) * 3 * (size_t)n)) != TB_OK) return s;
    TB_CK(cudaMemcpyAsync(ob.dev, F, sizeof(double) * 3 * (size_t)n, cudaMemcpyDeviceToDevice, st));
    return merge(run, out_finish(ob, st));
}

tb_status tb_csc_loop(tb_handle* h, int32_t K, const double* z, const double* w, double g_s, const double* gamma,
                      const double* q_ref, const double* dq_init, const tb_csc_opts* copts,
                      const tb_solve_opts* opts, double* q_out, double* dq_out, tb_csc_stats* stats,
                      void* stream) {
    if (!h || !gamma || !q_ref || !copts || !q_out || !dq_out) return TB_ERR_INVALID_ARG;
    if (copts->max_scf < 1 || !(copts->scf_tol > 0.0) || !(copts->mix > 0.0 && copts->mix <= 1.0))
        return TB_ERR_INVALID_ARG;
    const auto t0 = std::chrono::steady_clock::now();
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    tb_status s;
    if ((s = check_opts(opts)) != TB_OK) return s;
    if ((s = check_shifts(K, z, opts)) != TB_OK) return s;
    if (!w || !std::isfinite(g_s)) return TB_ERR_INVALID_ARG;
    if ((s = ensure_H0(h, st)) != TB_OK) return s;
    Cleanup cl;
    cl.st = st;
    const int n = h->n_atoms;
    const double *gd = nullptr, *qrd = nullptr;
    if ((s = device_view(cl, gamma, (size_t)n * n, &gd, st)) != TB_OK) return s;
    if ((s = device_view(cl, q_ref, (size_t)n, &qrd, st)) != TB_OK) return s;
    double *dq_in, *dq_next, *V, *q;
    unsigned long long* res_bits;
    if ((s = dalloc(cl, &dq_in, (size_t)n)) != TB_OK) return s;
    if ((s = dalloc(cl, &dq_next, (size_t)n)) != TB_OK) return s;
    if ((s = dalloc(cl, &V, (size_t)n)) != TB_OK) return s;
    if ((s = dalloc(cl, &q, (size_t)n)) != TB_OK) return s;
    if ((s = dalloc(cl, &res_bits, 1)) != TB_OK) return s;
    if (dq_init) {
        TB_CK(cudaMemcpyAsync(dq_in, dq_init, sizeof(double) * n, cudaMemcpyDefault, st));
    } else {
        TB_CK(cudaMemsetAsync(dq_in, 0, sizeof(double) * n, st));
    }
    tb_csc_stats cs{};
    bool cocg_unconverged = false;
    double res = 0.0;
    int m = 0;
    for (m = 1; m <= copts->max_scf; ++m) {
        launch_csc_potential(gd, dq_in, n, V, st);
        launch_csc_hamiltonian(h->ds, h->H0, V, st);
        TB_CK(cudaGetLastError());
        tb_stats ts{};
        const tb_status run = mulliken_atoms_device(h, K, z, w, g_s, opts, q, &ts, st);
        if (run != TB_OK && run != TB_ERR_NOT_CONVERGED) return run;
        if (run == TB_ERR_NOT_CONVERGED) cocg_unconverged = true;
        cs.outer_iterations += ts.outer_iterations;
        cs.inner_iterations += ts.inner_iterations;
        TB_CK(cudaMemsetAsync(res_bits, 0, sizeof(unsigned long long), st));
        launch_csc_mix(q, qrd, dq_in, dq_next, copts->mix, n, res_bits, st);
        TB_CK(cudaGetLastError());
        unsigned long long bits = 0;
        TB_CK(cudaMemcpyAsync(&bits, res_bits, sizeof(bits), cudaMemcpyDeviceToHost, st));
        TB_CK(cudaStreamSynchronize(st));
        std::memcpy(&res, &bits, sizeof(res));
        if (!std::isfinite(res)) return TB_ERR_BREAKDOWN;
        if (res <= copts->scf_tol || m == copts->max_scf) break;
        std::swap(dq_in, dq_next);
    }
    cs.iterations = std::min(m, copts->max_scf);
    cs.residual = res;
    TB_CK(cudaMemcpyAsync(dq_out, dq_in, sizeof(double) * n, cudaMemcpyDefault, st));
    TB_CK(cudaMemcpyAsync(q_out, q, sizeof(double) * n, cudaMemcpyDefault, st));
    TB_CK(cudaStreamSynchronize(st));
    cs.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (stats) *stats = cs;
    return (res <= copts->scf_tol && !cocg_unconverged) ? TB_OK : TB_ERR_NOT_CONVERGED;
}

tb_status tb_lanczos_green_batch(int32_t R, const double* a, const double* b, const double* norm, int32_t n_steps,
                                 int32_t K, const double* z, double* G_out, void* stream) {
    if (R < 1 || !a || !b || !norm || !z || !G_out || n_steps < 1 || K < 1) return TB_ERR_INVALID_ARG;
    for (int k = 0; k < 2 * K; ++k)
        if (!std::isfinite(z[k])) return TB_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Cleanup cl;
    cl.st = st;
    tb_status s;
    const double *ad = nullptr, *bd = nullptr, *nd = nullptr, *zd = nullptr;
    if ((s = device_view(cl, a, (size_t)R * n_steps, &ad, st)) != TB_OK) return s;
    if ((s = device_view(cl, b, (size_t)R * (n_steps + 1), &bd, st)) != TB_OK) return s;
    if ((s = device_view(cl, norm, (size_t)R, &nd, st)) != TB_OK) return s;
    if ((s = device_view(cl, z, (size_t)2 * K, &zd, st)) != TB_OK) return s;
    if (!is_device_ptr(norm))
        for (int r = 0; r < R; ++r)
            if (!std::isfinite(norm[r])) return TB_ERR_INVALID_ARG;
    OutBuf ob;
    if ((s = out_prepare(cl, ob, G_out, sizeof(double2) * (size_t)R * K)) != TB_OK) return s;
    launch_lanczos_green(ad, bd, nd, R, n_steps, K, reinterpret_cast<const double2*>(zd),
                         static_cast<double2*>(ob.dev), st);
    TB_CK(cudaGetLastError());
    return out_finish(ob, st);
}

tb_status tb_lanczos_green(const double* a, const double* b, double norm, int32_t n_steps, int32_t K,
                           const double* z, double* G_out, void* stream) {
    if (!std::isfinite(norm)) return TB_ERR_INVALID_ARG;
    return tb_lanczos_green_batch(1, a, b, &norm, n_steps, K, z, G_out, stream);
}

tb_status tb_generalized_lanczos_batch(tb_handle* h, int32_t R, const int32_t* cols, int32_t n_steps,
                                       const tb_solve_opts* opts, double* a, double* b, double* norm,
                                       void* stream) {
    if (!h || !a || !b || !norm || n_steps < 1) return TB_ERR_INVALID_ARG;
    tb_status s;
    if ((s = check_opts(opts)) != TB_OK) return s;
    if ((s = check_cols(h, R, cols)) != TB_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int npad = h->ds.npad;
    const int P = std::min(opts->panel ? opts->panel : 64, next_pow2(R));
    Cleanup cl_out;
    cl_out.st = st;
    OutBuf oa, ob, on;
    if ((s = out_prepare(cl_out, oa, a, sizeof(double) * (size_t)R * n_steps)) != TB_OK) return s;
    if ((s = out_prepare(cl_out, ob, b, sizeof(double) * (size_t)R * (n_steps + 1))) != TB_OK) return s;
    if ((s = out_prepare(cl_out, on, norm, sizeof(double) * (size_t)R)) != TB_OK) return s;
    View v = whole_view(h);
    for (int c0 = 0; c0 < R; c0 += P) {
        const int ncols = std::min(P, R - c0);
        Cleanup cl;
        cl.st = st;
        PanelDev p;
        p.P = P;
        p.K = 1;
        p.npad = npad;
        p.grid = max_grid();
        p.inner_tol = opts->inner_tol;
        p.mixed = opts->precision == TB_MIXED ? 1 : 0;
        p.inner_lo_tol = opts->inner_lo_tol;
        if ((s = alloc_inner_workspace(cl, p, st)) != TB_OK) return s;
        const size_t nv = (size_t)npad * P;
        double2 *U, *Uprev, *Wv;
        if ((s = dalloc(cl, &U, nv)) != TB_OK) return s;
        if ((s = dalloc(cl, &Uprev, nv)) != TB_OK) return s;
        if ((s = dalloc(cl, &Wv, nv)) != TB_OK) return s;
        // this panel's rows of the outputs ([R][n_steps], [R][n_steps + 1], [R])
        double* ad = static_cast<double*>(oa.dev) + (size_t)c0 * n_steps;
        double* bd = static_cast<double*>(ob.dev) + (size_t)c0 * (n_steps + 1);
        double* nd = static_cast<double*>(on.dev) + c0;
        double *ap, *bp, *np_;
        if ((s = dalloc(cl, &ap, (size_t)P * n_steps)) != TB_OK) return s;
        if ((s = dalloc(cl, &bp, (size_t)P * (n_steps + 1))) != TB_OK) return s;
        if ((s = dalloc(cl, &np_, (size_t)P)) != TB_OK) return s;
        std::vector<ColState> colh(P);
        for (int c = 0; c < P; ++c) {
            std::memset(&colh[c], 0, sizeof(ColState));
            colh[c].active = c < ncols ? 1 : 0;
            colh[c].row = c < ncols ? h->orb2pad_h[cols[c0 + c]] : -1;
        }
        TB_CK(cudaMemcpyAsync(p.col, colh.data(), sizeof(ColState) * P, cudaMemcpyHostToDevice, st));
        TB_CK(cudaMemsetAsync(p.inner, 0, 2 * P * sizeof(InnerState), st));
        if (p.mixed) {
            TB_CK(cudaMemsetAsync(p.inner32, 0, sizeof(InnerState) * 3 * 2 * P, st));
            TB_CK(cudaMemsetAsync(p.acc32, 0, sizeof(double) * 8 * P, st));
        }
        TB_CK(cudaMemsetAsync(p.flags, 0, NFLAGS * sizeof(int), st));
        TB_CK(cudaMemsetAsync(p.counter, 0, sizeof(unsigned) * (1 + MAX_GROUPS), st));
        TB_CK(cudaMemsetAsync(Uprev, 0, sizeof(double2) * nv, st));
        TB_CK(cudaMemsetAsync(ap, 0, sizeof(double) * P * n_steps, st));
        TB_CK(cudaMemsetAsync(bp, 0, sizeof(double) * P * (n_steps + 1), st));
        InnerCtx ic;
        if ((s = inner_ctx_init(v, opts, ic)) != TB_OK) return s;
        // u^0 = S^-1 e_j / sqrt(e_j^T S^-1 e_j); inner solves take the right-hand
        // side in Rcur (refinement) and Rin (FP64 CG), the solution in Rp
        launch_panel_init(h->ds, p, st);
        if ((s = inner_solve(v, p, p.Rcur, opts->inner_max_iter, ic, st)) != TB_OK) return s;
        launch_lz_start(p, p.Rp, U, np_, st);
        for (int n = 0; n < n_steps; ++n) {
            launch_lz_spmv(h->ds, h->ds.H, U, p.W, P, st);                        // H u^n
            launch_lz_dot(p, U, p.W, ap + n, n_steps, 0, st);                     // a_n = u^T H u
            TB_CK(cudaMemcpyAsync(p.Rin, p.W, sizeof(double2) * nv, cudaMemcpyDeviceToDevice, st));
            TB_CK(cudaMemcpyAsync(p.Rcur, p.W, sizeof(double2) * nv, cudaMemcpyDeviceToDevice, st));
            if ((s = inner_solve(v, p, p.Rcur, opts->inner_max_iter, ic, st)) != TB_OK) return s;  // S^-1 H u^n
            launch_lz_combine(p, p.Rp, U, Uprev, Wv, ap + n, bp + n, n_steps, n_steps + 1, st);
            launch_lz_spmv(h->ds, h->ds.S, Wv, p.W, P, st);                      // S w
            launch_lz_dot(p, Wv, p.W, bp + n + 1, n_steps + 1, 1, st);            // b_{n+1} = ||w||_S
            launch_lz_scale(p, Wv, U, Uprev, bp + n + 1, n_steps + 1, st);
            TB_CK(cudaGetLastError());
        }
        if (v.flags_host[0] & ERR_NOT_SPD) return TB_ERR_S_NOT_SPD;
        TB_CK(cudaMemcpyAsync(ad, ap, sizeof(double) * ncols * n_steps, cudaMemcpyDeviceToDevice, st));
        TB_CK(cudaMemcpyAsync(bd, bp, sizeof(double) * ncols * (n_steps + 1), cudaMemcpyDeviceToDevice, st));
        TB_CK(cudaMemcpyAsync(nd, np_, sizeof(double) * ncols, cudaMemcpyDeviceToDevice, st));
        TB_CK(cudaStreamSynchronize(st));
    }
    tb_status fin = out_finish(oa, st);
    if (fin == TB_OK) fin = out_finish(ob, st);
    if (fin == TB_OK) fin = out_finish(on, st);
    return fin;
}

tb_status tb_generalized_lanczos(tb_handle* h, int32_t j, int32_t n_steps, double inner_tol, double* a,
                                 double* b, double* norm, void* stream) {
    if (!h || j < 0 || j >= h->n_orb) return TB_ERR_INVALID_ARG;
    tb_solve_opts o;
    tb_default_opts(&o);
    o.inner_tol = inner_tol > 0.0 ? inner_tol : 1e-13;
    const int32_t col = j;
    return tb_generalized_lanczos_batch(h, 1, &col, n_steps, &o, a, b, norm, stream);
}

}  // extern "C"

// Carves aligned pieces out of the fixed scratch; fails when it would overrun.
struct ScratchCarver {
    unsigned char* base;
    size_t used = 0, cap;
    bool ok = true;
    ScratchCarver(unsigned char* b, size_t c) : base(b), cap(c) {}
    template <class T>
    T* take(size_t count) {
        const size_t bytes = ((count * sizeof(T) + 255) / 256) * 256;
        if (used + bytes > cap) {
            ok = false;
            return nullptr;
        }
        T* r = reinterpret_cast<T*>(base + used);
        used += bytes;
        return r;
    }
};

extern "C" {

tb_status tb_generalized_lanczos_noalloc(tb_handle* h, int32_t j, int32_t n_steps, double inner_tol, double* a,
                                         double* b, double* norm, void* stream) {
    if (!h || !a || !b || !norm || n_steps < 1 || j < 0 || j >= h->n_orb) return TB_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int npad = h->ds.npad;
    PanelDev p;
    p.P = 1;
    p.K = 1;
    p.npad = npad;
    p.grid = max_grid();
    p.inner_tol = inner_tol > 0.0 ? inner_tol : 1e-13;
    // size check before any device work: everything must fit in the fixed array
    ScratchCarver dry(nullptr, TB_NOALLOC_SCRATCH_BYTES);
    for (int v = 0; v < 10; ++v) dry.take<double2>(npad);
    dry.take<ColState>(1);
    dry.take<InnerState>(2);
    dry.take<double>((size_t)p.grid * 4);
    dry.take<double>((size_t)MAX_GROUPS * 4);
    dry.take<unsigned>(1 + MAX_GROUPS);
    dry.take<int>(NFLAGS);
    dry.take<double>(n_steps);
    dry.take<double>((size_t)n_steps + 1);
    dry.take<double>(1);
    if (!dry.ok) return TB_ERR_TOO_LARGE;
    // the handle's device must be current: the scratch address and the
    // kernels were placed there by tb_create
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return TB_ERR_CUDA;
    }
    if (dev != h->device || !h->noalloc_base) return TB_ERR_INVALID_ARG;
    tb_status s = TB_OK;
    ScratchCarver sc(h->noalloc_base, TB_NOALLOC_SCRATCH_BYTES);
    double2** vecs[] = {&p.Rcur, &p.Rprev, &p.Rp, &p.W, &p.Rin, &p.Pin, &p.Sin};
    for (double2** v : vecs) *v = sc.take<double2>(npad);
    double2* U = sc.take<double2>(npad);
    double2* Uprev = sc.take<double2>(npad);
    double2* Wv = sc.take<double2>(npad);
    p.col = sc.take<ColState>(1);
    p.inner = sc.take<InnerState>(2);
    p.partials = sc.take<double>((size_t)p.grid * 4);
    p.partials2 = sc.take<double>((size_t)MAX_GROUPS * 4);
    p.counter = sc.take<unsigned>(1 + MAX_GROUPS);
    p.flags = sc.take<int>(NFLAGS);
    double* ad = sc.take<double>(n_steps);
    double* bd = sc.take<double>((size_t)n_steps + 1);
    double* nd = sc.take<double>(1);
    if (!sc.ok) return TB_ERR_TOO_LARGE;
    // the array keeps the previous call's contents: clear everything that
    // the step loop reads before writing
    ColState cs;
    std::memset(&cs, 0, sizeof(cs));
    cs.active = 1;
    cs.row = h->orb2pad_h[j];
    TB_CK(cudaMemcpyAsync(p.col, &cs, sizeof(cs), cudaMemcpyHostToDevice, st));
    TB_CK(cudaMemsetAsync(p.inner, 0, 2 * sizeof(InnerState), st));
    TB_CK(cudaMemsetAsync(p.flags, 0, NFLAGS * sizeof(int), st));
    TB_CK(cudaMemsetAsync(p.counter, 0, sizeof(unsigned) * (1 + MAX_GROUPS), st));
    TB_CK(cudaMemsetAsync(Uprev, 0, sizeof(double2) * npad, st));
    TB_CK(cudaMemsetAsync(ad, 0, sizeof(double) * n_steps, st));
    TB_CK(cudaMemsetAsync(bd, 0, sizeof(double) * (n_steps + 1), st));
    int pred = 64;
    int64_t inner_total = 0;
    const int inner_max = 1000;
    View hv = whole_view(h);
    launch_panel_init(h->ds, p, st);
    if ((s = inner_cg(hv, p, inner_max, pred, inner_total, st)) != TB_OK) return s;
    launch_lz_start(p, p.Rp, U, nd, st);
    for (int n = 0; n < n_steps; ++n) {
        launch_lz_spmv(h->ds, h->ds.H, U, p.W, 1, st);
        launch_lz_dot(p, U, p.W, ad + n, 1, 0, st);
        TB_CK(cudaMemcpyAsync(p.Rin, p.W, sizeof(double2) * npad, cudaMemcpyDeviceToDevice, st));
        if ((s = inner_cg(hv, p, inner_max, pred, inner_total, st)) != TB_OK) return s;
        launch_lz_combine(p, p.Rp, U, Uprev, Wv, ad + n, bd + n, 1, 1, st);
        launch_lz_spmv(h->ds, h->ds.S, Wv, p.W, 1, st);
        launch_lz_dot(p, Wv, p.W, bd + n + 1, 1, 1, st);
        launch_lz_scale(p, Wv, U, Uprev, bd + n + 1, 1, st);
        TB_CK(cudaGetLastError());
    }
    if (h->flags_host[0] & ERR_NOT_SPD) return TB_ERR_S_NOT_SPD;
    const bool ad_dev = is_device_ptr(a), bd_dev = is_device_ptr(b), nd_dev = is_device_ptr(norm);
    TB_CK(cudaMemcpyAsync(a, ad, sizeof(double) * n_steps, ad_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
    TB_CK(cudaMemcpyAsync(b, bd, sizeof(double) * (n_steps + 1), bd_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
    TB_CK(cudaMemcpyAsync(norm, nd, sizeof(double), nd_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
    TB_CK(cudaStreamSynchronize(st));
    return TB_OK;
}

}  // extern "C"
