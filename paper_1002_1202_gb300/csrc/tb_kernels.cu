// CUDA kernels of the generalized shifted COCG hot path (sm_103a).
//
// Data layout (device, HBM):
//   * S and H: block-sparse rows over atoms, every block padded to 4x4
//     (row-major doubles), block row I covering padded orbitals 4I..4I+3;
//   * panel vectors: [npad][P] complex doubles (double2), the P right-hand
//     sides of a panel interleaved per orbital row, so one atom's 4 rows of a
//     panel are 4*P*16 contiguous bytes and a CTA's loads are coalesced along
//     the column index.
//
// Reductions are deterministic: each CTA writes per-column partial sums, the
// last CTA to arrive (atomic ticket) adds the partials in CTA order and
// turns them into the step's scalars.  Grid sizes are fixed per launch, so
// the summation order never changes between runs.
#include "tb_internal.h"

#include <math.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <thread>
#include <type_traits>
#include <cstdlib>
#include <vector>

namespace tb {

namespace {

__device__ __forceinline__ double2 cmk(double r, double i) { return make_double2(r, i); }
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return cmk(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return cmk(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return cmk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// complex division by Smith's method (no intermediate overflow of |b|^2)
__device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
    if (fabs(b.x) >= fabs(b.y)) {
        double r = b.y / b.x, den = b.x + b.y * r;
        return cmk((a.x + a.y * r) / den, (a.y - a.x * r) / den);
    }
    double r = b.x / b.y, den = b.y + b.x * r;
    return cmk((a.x * r + a.y) / den, (a.y * r - a.x) / den);
}
__device__ __forceinline__ double cabs2(double2 a) { return hypot(a.x, a.y); }

// Double-float products for FP64-accurate SpMVs on FP32 units (mixed path).
// A value is carried as hi + lo (two FP32 numbers, |lo| <= ulp(hi)/2).
// acc += s * x: the rounded product p = sh*xh and its exact error
// fma(sh, xh, -p) (Dekker / Ogita-Rump-Oishi error-free transformations),
// the cross terms sh*xl + sl*xh (sl*xl is below the working accuracy), and a
// two-sum of hi + p whose error goes to lo.  The _rn intrinsics keep the
// compiler from contracting these steps into FMAs, which would break the
// error terms.  Relative accuracy of a sum of n products ~ n * 2^-46.
// df_mac2 does this for a (re, im) pair that shares s, in packed FP32
// instructions (two lanes each, round-to-nearest per lane: each lane
// computes exactly the scalar sequence); a - b is a + (-b), which is exact.
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ void df_mac2(float2& hi, float2& lo, float sh, float sl, float2 xh, float2 xl) {
    const float2 s2h = make_float2(sh, sh), s2l = make_float2(sl, sl);
    const float2 pr = __fmul2_rn(s2h, xh);
    float2 e = __ffma2_rn(s2h, xh, neg2(pr));
    e = __ffma2_rn(s2h, xl, e);
    e = __ffma2_rn(s2l, xh, e);
    const float2 t = __fadd2_rn(hi, pr);
    const float2 bp = __fadd2_rn(t, neg2(hi));
    const float2 err = __fadd2_rn(__fadd2_rn(hi, neg2(__fadd2_rn(t, neg2(bp)))), __fadd2_rn(pr, neg2(bp)));
    hi = t;
    lo = __fadd2_rn(lo, __fadd2_rn(err, e));
}

// complex double -> (re_hi, im_hi, re_lo, im_lo): the hi and lo pairs are
// the two float2 operands of df_mac2
__device__ __forceinline__ float4 df_split(double2 v) {
    const float rh = (float)v.x, ih = (float)v.y;
    return make_float4(rh, ih, (float)(v.x - (double)rh), (float)(v.y - (double)ih));
}

// Sum NV per-thread values over the threads of a CTA that share a column
// (column = tid % P).  Result for column c (< P) in smem[q*THREADS + c].
template <int NV>
__device__ void block_reduce_cols(const double (&v)[NV], int P, double* smem) {
    const int tid = threadIdx.x;
#pragma unroll
    for (int q = 0; q < NV; ++q) smem[q * THREADS + tid] = v[q];
    __syncthreads();
    for (int s = (THREADS / P) / 2; s >= 1; s >>= 1) {
        if (tid < s * P) {
#pragma unroll
            for (int q = 0; q < NV; ++q) smem[q * THREADS + tid] += smem[q * THREADS + tid + s * P];
        }
        __syncthreads();
    }
}

// Grid-wide per-column sums, as a deterministic two-level tree.  Each CTA
// writes its block sums; the last CTA of every group of RED_GROUP CTAs
// (atomic ticket) adds its group's sums in CTA order; the last group
// reducer adds the group sums in group order.  Returns true in that final
// CTA, whose threads tid < P then find the total of column tid in
// smem[q*THREADS + tid].  No CTA waits on another.
template <int NV>
__device__ bool grid_reduce_cols(const double (&v)[NV], int P, const PanelDev& p, double* smem) {
    __shared__ int s_last;
    const int tid = threadIdx.x;
    const int nblk = gridDim.x;
    const int ngrp = (nblk + RED_GROUP - 1) / RED_GROUP;
    const int grp = blockIdx.x / RED_GROUP;
    const int gbeg = grp * RED_GROUP;
    const int gsize = min(RED_GROUP, nblk - gbeg);
    block_reduce_cols<NV>(v, P, smem);
    if (tid < P) {
#pragma unroll
        for (int q = 0; q < NV; ++q) p.partials[((size_t)blockIdx.x * NV + q) * P + tid] = smem[q * THREADS + tid];
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) s_last = (atomicAdd(&p.counter[1 + grp], 1u) == (unsigned)gsize - 1);
    __syncthreads();
    if (!s_last) return false;
    __threadfence();
    const int c = tid % P, g = tid / P, G = THREADS / P;
    double acc[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) acc[q] = 0.0;
    for (int b = gbeg + g; b < gbeg + gsize; b += G) {
#pragma unroll
        for (int q = 0; q < NV; ++q) acc[q] += __ldcg(&p.partials[((size_t)b * NV + q) * P + c]);
    }
    __syncthreads();
    block_reduce_cols<NV>(acc, P, smem);
    if (tid == 0) p.counter[1 + grp] = 0u;
    if (ngrp == 1) return true;
    if (tid < P) {
#pragma unroll
        for (int q = 0; q < NV; ++q) p.partials2[((size_t)grp * NV + q) * P + tid] = smem[q * THREADS + tid];
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) s_last = (atomicAdd(&p.counter[0], 1u) == (unsigned)ngrp - 1);
    __syncthreads();
    if (!s_last) return false;
    __threadfence();
#pragma unroll
    for (int q = 0; q < NV; ++q) acc[q] = 0.0;
    for (int b = g; b < ngrp; b += G) {
#pragma unroll
        for (int q = 0; q < NV; ++q) acc[q] += __ldcg(&p.partials2[((size_t)b * NV + q) * P + c]);
    }
    __syncthreads();
    block_reduce_cols<NV>(acc, P, smem);
    if (tid == 0) p.counter[0] = 0u;
    return true;
}

// ---------------------------------------------------------------------------
// ASED Hamiltonian (Section 2.2, Eq. Hap-1) built from S on the device.
// ---------------------------------------------------------------------------
__global__ void k_ased_build(int n_atoms, const int* __restrict__ brow, const int* __restrict__ bcol,
                             const double* __restrict__ S, double* __restrict__ H,
                             const double* __restrict__ eps, double K) {
    for (int I = blockIdx.x * blockDim.x + threadIdx.x; I < n_atoms; I += gridDim.x * blockDim.x) {
        for (int b = brow[I]; b < brow[I + 1]; ++b) {
            const int J = bcol[b];
            for (int a = 0; a < 4; ++a) {
                for (int c = 0; c < 4; ++c) {
                    double h;
                    if (I == J) h = (a == c) ? eps[4 * I + a] : 0.0;   // on-site level
                    else h = K * 0.5 * (eps[4 * I + a] + eps[4 * J + c]) * S[16 * (size_t)b + 4 * a + c];
                    H[16 * (size_t)b + 4 * a + c] = h;
                }
            }
        }
    }
}

// hi + lo FP32 split of a FP64 array
__global__ void k_split_f64(const double* __restrict__ v, float* __restrict__ hi, float* __restrict__ lo, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float h = (float)v[i];
        hi[i] = h;
        lo[i] = (float)(v[i] - (double)h);
    }
}

// r_0 = b = e_j, r_{-1} = 0, inner right-hand side = b
// out[b] = in[b]^T for every 4 x 4 FP32 block (the Chebyshev step reads the
// columns of S_IJ as rows)
__global__ void k_transpose_blocks(const float* __restrict__ in, float* __restrict__ out, long long nb) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < 16 * nb;
         i += (long long)gridDim.x * blockDim.x) {
        const long long b = i >> 4;
        const int a = (int)(i >> 2) & 3, e = (int)i & 3;
        out[16 * b + 4 * e + a] = in[i];
    }
}

// The compact FP32 blocks of a system with s-only atoms (see DevSystem):
// one thread per block row I, its blocks in order.
__global__ void k_compact_blocks(int n_atoms, const int* __restrict__ brow, const int* __restrict__ bcol,
                                 const unsigned char* __restrict__ norb, const float* __restrict__ S32,
                                 const int2* __restrict__ bmeta, float* __restrict__ out) {
    for (int I = blockIdx.x * blockDim.x + threadIdx.x; I < n_atoms; I += gridDim.x * blockDim.x) {
        const int ni = norb[I];
        for (int b = brow[I]; b < brow[I + 1]; ++b) {
            const int nj = norb[bcol[b]];
            const float* S = S32 + 16 * (size_t)b;
            float* o = out + 4 * (size_t)(bmeta[b].y & 0x7fffffff);
            if (ni == 4 && nj == 4) {
                for (int e = 0; e < 4; ++e)
                    for (int a = 0; a < 4; ++a) o[4 * e + a] = S[4 * a + e];
            } else if (ni == 4) {
                for (int a = 0; a < 4; ++a) o[a] = S[4 * a];
            } else if (nj == 4) {
                for (int e = 0; e < 4; ++e) o[e] = S[e];
            } else {
                o[0] = S[0];
                o[1] = o[2] = o[3] = 0.f;
            }
        }
    }
}

__global__ void k_panel_init(PanelDev p) {
    const long long items = (long long)p.npad * p.P;
    for (long long idx = blockIdx.x * (long long)THREADS + threadIdx.x; idx < items;
         idx += (long long)gridDim.x * THREADS) {
        const int c = (int)(idx % p.P), i = (int)(idx / p.P);
        const double2 v = cmk(i == p.col[c].row ? 1.0 : 0.0, 0.0);
        p.Rcur[idx] = v;
        p.Rin[idx] = v;
        p.Rprev[idx] = cmk(0.0, 0.0);
    }
}

// ---------------------------------------------------------------------------
// a1 + a2: q = A(z_s) r'_n = z_s S r'_n - H r'_n in one pass over the blocks,
// A p_n = q + (beta_{n-1}/alpha_{n-1}) (r_{n-1} - r_n), mu = r'_n^T A p_n,
// alpha_n = rho_n / mu (Eqs. CGp:p, CGp:r and the alpha_n of Section 3.3).
// Pending seed-switch scales of r_n, r'_n, r_{n-1} are applied on the fly.
// SX (mixed path): S r'_n is taken as r_n - res, res = r_n - S r'_n being
// the refinement's last double-float residual (in Rin), so only H r'_n is
// formed here -- half the double-float products.
// ---------------------------------------------------------------------------
// One block row of a double-float SpMV (M = Mh + Ml, FP32 hi / lo blocks,
// times the split r') with exact orbital counts (systems with s-only atoms):
// only the ni real rows of atom I and, per block, the real rows of the
// column atom (one for an s atom, read with the column S[.][0]) -- the
// padded entries would only add exact zeros.
__device__ __forceinline__ void df_row_ragged(const DevSystem& s, const float* __restrict__ Mh,
                                              const float* __restrict__ Ml, int I, int ni,
                                              const float4* __restrict__ RpS, int P, int c, float2 (&hi)[4],
                                              float2 (&lo)[4]) {
    for (int bb = s.brow[I]; bb < s.brow[I + 1]; ++bb) {
        const int2 m = __ldg(s.bmeta + bb);
        const float4* xr = RpS + (size_t)4 * m.x * P + c;
        if (m.y >= 0) {
            const float4 x[4] = {xr[0], xr[P], xr[2 * P], xr[3 * P]};
            const float4* Bh = reinterpret_cast<const float4*>(Mh + 16 * (size_t)bb);
            const float4* Bl = reinterpret_cast<const float4*>(Ml + 16 * (size_t)bb);
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                if (a >= ni) break;
                const float4 v4h = __ldg(Bh + a), v4l = __ldg(Bl + a);
                const float vh[4] = {v4h.x, v4h.y, v4h.z, v4h.w}, vl[4] = {v4l.x, v4l.y, v4l.z, v4l.w};
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    df_mac2(hi[a], lo[a], vh[e], vl[e], make_float2(x[e].x, x[e].y), make_float2(x[e].z, x[e].w));
            }
        } else {
            const float4 x0 = xr[0];
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                if (a >= ni) break;
                df_mac2(hi[a], lo[a], __ldg(Mh + 16 * (size_t)bb + 4 * a), __ldg(Ml + 16 * (size_t)bb + 4 * a),
                        make_float2(x0.x, x0.y), make_float2(x0.z, x0.w));
            }
        }
    }
}

template <bool DF, bool SX = false, bool RAG = false>
__global__ void __launch_bounds__(THREADS) k_outer_spmm(DevSystem s, PanelDev p) {
    __shared__ double smem[2 * THREADS];
    const int P = p.P;
    const int c = threadIdx.x % P;
    const ColState cs = p.col[c];
    const bool act = cs.active != 0;
    const double2 sc = cs.sc_cur, scp = cs.sc_prev;
    const double2 coef = act ? cdiv(cs.beta_prev, cs.alpha_prev) : cmk(0.0, 0.0);
    double mu[2] = {0.0, 0.0};
    const long long items = (long long)s.n_atoms * P;
    if (act) {
        for (long long idx = blockIdx.x * (long long)THREADS + threadIdx.x; idx < items;
             idx += (long long)gridDim.x * THREADS) {
            const int I = (int)(idx / P);
            double2 aS[4], aH[4];
            if (DF) {
                // double-float products: S_hi/S_lo, H_hi/H_lo times the split r',
                // the real and imaginary parts in the two lanes of packed FP32 ops
                float2 sh[4], sl[4], hh[4], hl[4];
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    sh[a] = sl[a] = hh[a] = hl[a] = make_float2(0.f, 0.f);
                }
                if (RAG) {
                    const int ni = s.norb[I];
                    df_row_ragged(s, s.H32hi, s.H32lo, I, ni, p.RpS, P, c, hh, hl);
                    if (!SX) df_row_ragged(s, s.S32, s.S32lo, I, ni, p.RpS, P, c, sh, sl);
                }
                for (int b = RAG ? s.brow[I + 1] : s.brow[I]; b < s.brow[I + 1]; ++b) {
                    const int J = s.bcol[b];
                    const float4* xr = p.RpS + (size_t)4 * J * P + c;
                    const float4 x[4] = {xr[0], xr[P], xr[2 * P], xr[3 * P]};
                    const float4* Sh = reinterpret_cast<const float4*>(s.S32 + 16 * (size_t)b);
                    const float4* Sl = reinterpret_cast<const float4*>(s.S32lo + 16 * (size_t)b);
                    const float4* Hh = reinterpret_cast<const float4*>(s.H32hi + 16 * (size_t)b);
                    const float4* Hl = reinterpret_cast<const float4*>(s.H32lo + 16 * (size_t)b);
#pragma unroll
                    for (int a = 0; a < 4; ++a) {
                        const float4 h4h = __ldg(Hh + a), h4l = __ldg(Hl + a);
                        const float hvh[4] = {h4h.x, h4h.y, h4h.z, h4h.w}, hvl[4] = {h4l.x, h4l.y, h4l.z, h4l.w};
                        if (!SX) {
                            const float4 s4h = __ldg(Sh + a), s4l = __ldg(Sl + a);
                            const float svh[4] = {s4h.x, s4h.y, s4h.z, s4h.w}, svl[4] = {s4l.x, s4l.y, s4l.z, s4l.w};
#pragma unroll
                            for (int e = 0; e < 4; ++e)
                                df_mac2(sh[a], sl[a], svh[e], svl[e], make_float2(x[e].x, x[e].y),
                                        make_float2(x[e].z, x[e].w));
                        }
#pragma unroll
                        for (int e = 0; e < 4; ++e)
                            df_mac2(hh[a], hl[a], hvh[e], hvl[e], make_float2(x[e].x, x[e].y),
                                    make_float2(x[e].z, x[e].w));
                    }
                }
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    if (SX) {
                        const size_t e = (size_t)(4 * I + a) * P + c;
                        aS[a] = csub(p.Rcur[e], p.Rin[e]);
                    } else {
                        aS[a] = cmk((double)sh[a].x + (double)sl[a].x, (double)sh[a].y + (double)sl[a].y);
                    }
                    aH[a] = cmk((double)hh[a].x + (double)hl[a].x, (double)hh[a].y + (double)hl[a].y);
                }
            } else {
#pragma unroll
                for (int a = 0; a < 4; ++a) { aS[a] = cmk(0.0, 0.0); aH[a] = cmk(0.0, 0.0); }
                for (int b = s.brow[I]; b < s.brow[I + 1]; ++b) {
                    const int J = s.bcol[b];
                    const double2* xr = p.Rp + (size_t)4 * J * P + c;
                    const double2 x0 = xr[0], x1 = xr[P], x2 = xr[2 * P], x3 = xr[3 * P];
                    const double2* Sb = reinterpret_cast<const double2*>(s.S + 16 * (size_t)b);
                    const double2* Hb = reinterpret_cast<const double2*>(s.H + 16 * (size_t)b);
#pragma unroll
                    for (int a = 0; a < 4; ++a) {
                        const double2 s01 = __ldg(Sb + 2 * a), s23 = __ldg(Sb + 2 * a + 1);
                        const double2 h01 = __ldg(Hb + 2 * a), h23 = __ldg(Hb + 2 * a + 1);
                        aS[a].x += s01.x * x0.x + s01.y * x1.x + s23.x * x2.x + s23.y * x3.x;
                        aS[a].y += s01.x * x0.y + s01.y * x1.y + s23.x * x2.y + s23.y * x3.y;
                        aH[a].x += h01.x * x0.x + h01.y * x1.x + h23.x * x2.x + h23.y * x3.x;
                        aH[a].y += h01.x * x0.y + h01.y * x1.y + h23.x * x2.y + h23.y * x3.y;
                    }
                }
            }
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                const size_t e = (size_t)(4 * I + a) * P + c;
                const double2 q = cmul(sc, csub(cmul(cs.zs, aS[a]), aH[a]));
                const double2 rc = cmul(sc, p.Rcur[e]);
                const double2 rpv = cmul(scp, p.Rprev[e]);
                const double2 Ap = cadd(q, cmul(coef, csub(rpv, rc)));
                p.W[e] = Ap;
                const double2 m = cmul(cmul(sc, p.Rp[e]), Ap);
                mu[0] += m.x;
                mu[1] += m.y;
            }
        }
    }
    if (grid_reduce_cols<2>(mu, P, p, smem)) {
        const int t = threadIdx.x;
        if (t < P && p.col[t].active) {
            const double2 m = cmk(smem[t], smem[THREADS + t]);
            const double2 rho = p.col[t].rho;
            if ((m.x == 0.0 && m.y == 0.0) || (rho.x == 0.0 && rho.y == 0.0) || !isfinite(m.x) ||
                !isfinite(m.y)) {
                atomicOr(&p.flags[0], ERR_BREAKDOWN);
                p.col[t].active = 0;
            } else {
                p.col[t].alpha = cdiv(rho, m);
            }
        }
    }
}

// r_{n+1} = r_n - alpha_n A p_n; r_n becomes r_{n-1}; the inner CG starts
// from b = r_{n+1}.
__global__ void k_outer_update(PanelDev p) {
    const int P = p.P;
    const int c = threadIdx.x % P;
    const ColState cs = p.col[c];
    if (!cs.active) return;
    const long long items = (long long)p.npad * P;
    for (long long idx = blockIdx.x * (long long)THREADS + threadIdx.x; idx < items;
         idx += (long long)gridDim.x * THREADS) {
        const double2 rc = cmul(cs.sc_cur, p.Rcur[idx]);
        const double2 rn = csub(rc, cmul(cs.alpha, p.W[idx]));
        p.Rprev[idx] = rc;
        p.Rcur[idx] = rn;
        p.Rin[idx] = rn;
    }
}

// ---------------------------------------------------------------------------
// a3 + a4: inner CG for S r' = r (Section 3.3), both real parts of every
// complex column, Chronopoulos-Gear form (one reduction per iteration):
//   w_i = S r_i, gamma_i = r_i.r_i, delta_i = w_i.r_i,
//   beta_i = gamma_i/gamma_{i-1}, alpha_i = gamma_i/(delta_i - beta_i gamma_i/alpha_{i-1}),
//   p_i = r_i + beta_i p_{i-1}, s_i = w_i + beta_i s_{i-1},
//   x_{i+1} = x_i + alpha_i p_i, r_{i+1} = r_i - alpha_i s_i,   x_0 = 0.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(THREADS) k_inner_spmv(DevSystem s, PanelDev p, int it) {
    __shared__ double smem[4 * THREADS];
    if (it > 0 && *(volatile int*)&p.flags[1] == 0) return;
    const int P = p.P;
    const int c = threadIdx.x % P;
    const bool act = p.col[c].active != 0;
    const bool live = act && !(p.inner[2 * c].conv && p.inner[2 * c + 1].conv && it > 0);
    double v[4] = {0.0, 0.0, 0.0, 0.0};   // gamma_re, gamma_im, delta_re, delta_im
    const long long items = (long long)s.n_atoms * P;
    if (live) {
        for (long long idx = blockIdx.x * (long long)THREADS + threadIdx.x; idx < items;
             idx += (long long)gridDim.x * THREADS) {
            const int I = (int)(idx / P);
            double2 acc[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) acc[a] = cmk(0.0, 0.0);
            for (int b = s.brow[I]; b < s.brow[I + 1]; ++b) {
                const int J = s.bcol[b];
                const double2* xr = p.Rin + (size_t)4 * J * P + c;
                const double2 x0 = xr[0], x1 = xr[P], x2 = xr[2 * P], x3 = xr[3 * P];
                const double2* Sb = reinterpret_cast<const double2*>(s.S + 16 * (size_t)b);
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    const double2 s01 = __ldg(Sb + 2 * a), s23 = __ldg(Sb + 2 * a + 1);
                    acc[a].x += s01.x * x0.x + s01.y * x1.x + s23.x * x2.x + s23.y * x3.x;
                    acc[a].y += s01.x * x0.y + s01.y * x1.y + s23.x * x2.y + s23.y * x3.y;
                }
            }
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                const size_t e = (size_t)(4 * I + a) * P + c;
                const double2 r = p.Rin[e];
                p.W[e] = acc[a];
                v[0] += r.x * r.x;
                v[1] += r.y * r.y;
                v[2] += acc[a].x * r.x;
                v[3] += acc[a].y * r.y;
            }
        }
    }
    if (grid_reduce_cols<4>(v, P, p, smem)) {
        const int t = threadIdx.x;
        int nact = 0;
        if (t < P) {
            const bool cact = p.col[t].active != 0;
            if (it == 0 && cact) p.col[t].rnorm = sqrt(smem[t] + smem[THREADS + t]);
            for (int part = 0; part < 2; ++part) {
                InnerState st = p.inner[2 * t + part];
                const double gam = smem[part * THREADS + t];
                const double del = smem[(2 + part) * THREADS + t];
                if (it == 0) {
                    st.bnorm2 = gam;
                    st.conv = (!cact || gam == 0.0) ? 1 : 0;
                }
                if (!st.conv) {
                    if (gam <= p.inner_tol * p.inner_tol * st.bnorm2) {
                        st.conv = 1;
                    } else {
                        const double beta = (it == 0) ? 0.0 : gam / st.gamma_prev;
                        const double den = del - ((it == 0) ? 0.0 : beta * gam / st.alpha);
                        if (!(den > 0.0)) {
                            atomicOr(&p.flags[0], ERR_NOT_SPD);
                            st.conv = 1;
                        } else {
                            st.alpha = gam / den;
                            st.beta = beta;
                            st.gamma_prev = gam;
                        }
                    }
                }
                nact += st.conv ? 0 : 1;
                p.inner[2 * t + part] = st;
            }
        }
        // count unconverged real columns
        __shared__ int s_cnt;
        if (t == 0) s_cnt = 0;
        __syncthreads();
        if (nact) atomicAdd(&s_cnt, nact);
        __syncthreads();
        if (t == 0) {
            p.flags[1] = s_cnt;
            if (s_cnt == 0) p.flags[3] = it;
        }
    }
}

__global__ void k_inner_update(PanelDev p, int it) {
    if (it > 0 && *(volatile int*)&p.flags[1] == 0) return;
    const int P = p.P;
    const int c = threadIdx.x % P;
    if (!p.col[c].active) return;
    const InnerState s0 = p.inner[2 * c], s1 = p.inner[2 * c + 1];
    if (s0.conv && s1.conv && it > 0) return;
    const long long items = (long long)p.npad * P;
    for (long long idx = blockIdx.x * (long long)THREADS + threadIdx.x; idx < items;
         idx += (long long)gridDim.x * THREADS) {
        const double2 r = p.Rin[idx], w = p.W[idx];
        double2 pv = (it == 0) ? cmk(0.0, 0.0) : p.Pin[idx];
        double2 sv = (it == 0) ? cmk(0.0, 0.0) : p.Sin[idx];
        double2 x = (it == 0) ? cmk(0.0, 0.0) : p.Rp[idx];
        double2 rn = r;
        if (!s0.conv) {
            pv.x = r.x + s0.beta * pv.x;
            sv.x = w.x + s0.beta * sv.x;
            x.x += s0.alpha * pv.x;
            rn.x = r.x - s0.alpha * sv.x;
        }
        if (!s1.conv) {
            pv.y = r.y + s1.beta * pv.y;
            sv.y = w.y + s1.beta * sv.y;
            x.y += s1.alpha * pv.y;
            rn.y = r.y - s1.alpha * sv.y;
        }
        p.Pin[idx] = pv;
        p.Sin[idx] = sv;
        p.Rp[idx] = x;
        p.Rin[idx] = rn;
    }
}

// ---------------------------------------------------------------------------
// Mixed-precision inner solve (TB_MIXED): r' = S^-1 b by iterative
// refinement.  x_0 = 0; round m computes res_m = b - S x_m in FP64, scales
// it to unit norm, solves S d = res_m / ||res_m|| in FP32 to relative
// inner_lo_tol (Chebyshev steps, k_inner32_cheb below, or CG), and sets
// x_{m+1} = x_m + ||res_m|| d in FP64, until ||res_m|| <= inner_tol ||b||
// per real column.  The unit scaling keeps the FP32 values away from
// underflow however small b or the residual are.  The FP32 CG reuses the
// Chronopoulos-Gear form of the FP64 one.
// ---------------------------------------------------------------------------
__device__ void refine_finish_counts(PanelDev& p, int nact) {
    __shared__ int s_cnt;
    if (threadIdx.x == 0) s_cnt = 0;
    __syncthreads();
    if (nact) atomicAdd(&s_cnt, nact);
    __syncthreads();
    if (threadIdx.x == 0) {
        p.flags[1] = s_cnt;
        p.flags[4] = s_cnt;
    }
}

// round 0: ||b||, x = 0
__global__ void __launch_bounds__(THREADS) k_refine_start(PanelDev p, const double2* __restrict__ b) {
    __shared__ double smem[2 * THREADS];
    const int P = p.P;
    const int c = threadIdx.x % P;
    const bool act = p.col[c].active != 0;
    double v[2] = {0.0, 0.0};
    const long long items = (long long)p.npad * P;
    if (act) {
        for (long long idx = blockIdx.x * (long long)THREADS + threadIdx.x; idx < items;
             idx += (long long)gridDim.x * THREADS) {
            const double2 bv = b[idx];
            p.Rp[idx] = cmk(0.0, 0.0);
            p.RpS[idx] = make_float4(0.f, 0.f, 0.f, 0.f);
            v[0] += bv.x * bv.x;
            v[1] += bv.y * bv.y;
        }
    }
    if (grid_reduce_cols<2>(v, P, p, smem)) {
        const int t = threadIdx.x;
        int nact = 0;
        if (t < P) {
            const bool cact = p.col[t].active != 0;
            if (cact) p.col[t].rnorm = sqrt(smem[t] + smem[THREADS + t]);
            for (int part = 0; part < 2; ++part) {
                const double b2 = smem[part * THREADS + t];
                p.inner[2 * t + part].bnorm2 = b2;
                InnerState st = p.inner32[2 * t + part];
                st.skip = (!cact || b2 == 0.0) ? 1 : 0;
                st.unscale = st.skip ? 0.0 : sqrt(b2);
                st.scale = st.skip ? 0.0 : 1.0 / st.unscale;
                p.inner32[2 * t + part] = st;
                nact += st.skip ? 0 : 1;
            }
        }
        refine_finish_counts(p, nact);
    }
}

// res = b - S x in FP64 (x = r') into Rin; columns already within inner_tol
// are marked to skip the next round, the others get scale = 1 / ||res||.
template <bool DF, bool RAG = false>
__global__ void __launch_bounds__(THREADS) k_refine_residual(DevSystem s, PanelDev p, const double2* __restrict__ b) {
    __shared__ double smem[2 * THREADS];
    const int P = p.P;
    const int c = threadIdx.x % P;
    const bool act = p.col[c].active != 0 && !(p.inner32[2 * c].skip && p.inner32[2 * c + 1].skip);
    double v[2] = {0.0, 0.0};
    const long long items = (long long)s.n_atoms * P;
    if (act) {
        for (long long idx = blockIdx.x * (long long)THREADS + threadIdx.x; idx < items;
             idx += (long long)gridDim.x * THREADS) {
            const int I = (int)(idx / P);
            double2 acc[4];
            if (DF) {
                float2 ah[4], al[4];
#pragma unroll
                for (int a = 0; a < 4; ++a) ah[a] = al[a] = make_float2(0.f, 0.f);
                if (RAG) df_row_ragged(s, s.S32, s.S32lo, I, s.norb[I], p.RpS, P, c, ah, al);
                for (int bb = RAG ? s.brow[I + 1] : s.brow[I]; bb < s.brow[I + 1]; ++bb) {
                    const int J = s.bcol[bb];
                    const float4* xr = p.RpS + (size_t)4 * J * P + c;
                    const float4 x[4] = {xr[0], xr[P], xr[2 * P], xr[3 * P]};
                    const float4* Sh = reinterpret_cast<const float4*>(s.S32 + 16 * (size_t)bb);
                    const float4* Sl = reinterpret_cast<const float4*>(s.S32lo + 16 * (size_t)bb);
#pragma unroll
                    for (int a = 0; a < 4; ++a) {
                        const float4 s4h = __ldg(Sh + a), s4l = __ldg(Sl + a);
                        const float svh[4] = {s4h.x, s4h.y, s4h.z, s4h.w}, svl[4] = {s4l.x, s4l.y, s4l.z, s4l.w};
#pragma unroll
                        for (int e = 0; e < 4; ++e)
                            df_mac2(ah[a], al[a], svh[e], svl[e], make_float2(x[e].x, x[e].y),
                                    make_float2(x[e].z, x[e].w));
                    }
                }
#pragma unroll
                for (int a = 0; a < 4; ++a)
                    acc[a] = cmk((double)ah[a].x + (double)al[a].x, (double)ah[a].y + (double)al[a].y);
            } else {
#pragma unroll
                for (int a = 0; a < 4; ++a) acc[a] = cmk(0.0, 0.0);
                for (int bb = s.brow[I]; bb < s.brow[I + 1]; ++bb) {
                    const int J = s.bcol[bb];
                    const double2* xr = p.Rp + (size_t)4 * J * P + c;
                    const double2 x0 = xr[0], x1 = xr[P], x2 = xr[2 * P], x3 = xr[3 * P];
                    const double2* Sb = reinterpret_cast<const double2*>(s.S + 16 * (size_t)bb);
#pragma unroll
                    for (int a = 0; a < 4; ++a) {
                        const double2 s01 = __ldg(Sb + 2 * a), s23 = __ldg(Sb + 2 * a + 1);
                        acc[a].x += s01.x * x0.x + s01.y * x1.x + s23.x * x2.x + s23.y * x3.x;
                        acc[a].y += s01.x * x0.y + s01.y * x1.y + s23.x * x2.y + s23.y * x3.y;
                    }
                }
            }
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                const size_t e = (size_t)(4 * I + a) * P + c;
                const double2 r = csub(b[e], acc[a]);
                p.Rin[e] = r;
                v[0] += r.x * r.x;
                v[1] += r.y * r.y;
            }
        }
    }
    if (grid_reduce_cols<2>(v, P, p, smem)) {
        const int t = threadIdx.x;
        int nact = 0;
        if (t < P) {
            const bool cact = p.col[t].active != 0;
            for (int part = 0; part < 2; ++part) {
                InnerState st = p.inner32[2 * t + part];
                if (!st.skip) {
                    const double r2 = smem[part * THREADS + t];
                    const double b2 = p.inner[2 * t + part].bnorm2;
                    if (!isfinite(r2)) {
                        atomicOr(&p.flags[0], ERR_INNER);
                        if (p.dbg) {
                            p.dbg[0] = -1.0; p.dbg[1] = 2 * t + part; p.dbg[2] = r2; p.dbg[3] = st.scale;
                            p.dbg[4] = b2; p.dbg[5] = st.bnorm2; p.dbg[6] = st.gamma_prev; p.dbg[7] = st.alpha;
                        }
                        st.skip = 1;
                    } else if (!cact || r2 <= p.inner_tol * p.inner_tol * b2 || r2 == 0.0) {
                        st.skip = 1;
                    }
                    st.unscale = st.skip ? 0.0 : sqrt(r2);
                    st.scale = st.skip ? 0.0 : 1.0 / st.unscale;
                }
                nact += st.skip ? 0 : 1;
                p.inner32[2 * t + part] = st;
            }
        }
        refine_finish_counts(p, nact);
    }
}

// FP32 right-hand side of the round: src * scale (0 for a skipped real
// column; columns with both parts skipped are left alone, no kernel of the
// round reads them).  cheb_gamma > 0: also the first Chebyshev iterate
// d_1 = gamma f into x32 (the next round makes Chebyshev corrections).
__global__ void k_refine_scale(PanelDev p, const double2* __restrict__ src, float cheb_gamma) {
    const int P = p.P;
    const int c = threadIdx.x % P;
    if (blockIdx.x == 0) {
        for (int q = threadIdx.x; q < 8 * P; q += THREADS) p.acc32[q] = 0.0;   // both CG sum slots
        if (threadIdx.x == 0) p.flags[7] = -1;                                  // no CG scalars yet
    }
    if (!p.col[c].active) return;
    const InnerState i0 = p.inner32[2 * c], i1 = p.inner32[2 * c + 1];
    if (i0.skip && i1.skip) return;
    const double s0 = i0.scale, s1 = i1.scale;
    const long long items = (long long)p.npad * P;
    for (long long idx = blockIdx.x * (long long)THREADS + threadIdx.x; idx < items;
         idx += (long long)gridDim.x * THREADS) {
        const double2 v = src[idx];
        const float2 f = make_float2((float)(v.x * s0), (float)(v.y * s1));
        p.r32[idx] = f;
        if (cheb_gamma > 0.f) p.x32[idx] = make_float2(cheb_gamma * f.x, cheb_gamma * f.y);
    }
}

// r' copied into the FP64 inner right-hand side slot and split for the
// double-float products (after an FP64 redo of a mixed inner solve)
__global__ void k_split_panel(PanelDev p) {
    const int P = p.P;
    const int c = threadIdx.x % P;
    if (!p.col[c].active) return;
    const long long items = (long long)p.npad * P;
    for (long long idx = blockIdx.x * (long long)THREADS + threadIdx.x; idx < items;
         idx += (long long)gridDim.x * THREADS)
        p.RpS[idx] = df_split(p.Rp[idx]);
}

// x += d / scale (FP32 correction added in FP64) for the columns that took the round
__global__ void k_refine_add(PanelDev p) {
    const int P = p.P;
    const int c = threadIdx.x % P;
    if (!p.col[c].active) return;
    const InnerState i0 = p.inner32[2 * c], i1 = p.inner32[2 * c + 1];
    const bool u0 = !i0.skip, u1 = !i1.skip;
    if (!u0 && !u1) return;
    const double f0 = u0 ? i0.unscale : 0.0, f1 = u1 ? i1.unscale : 0.0;
    const long long items = (long long)p.npad * P;
    for (long long idx = blockIdx.x * (long long)THREADS + threadIdx.x; idx < items;
         idx += (long long)gridDim.x * THREADS) {
        const float2 d = p.x32[idx];
        double2 x = p.Rp[idx];
        // a non-finite correction is dropped: the next round starts again
        // from the FP64 residual
        if (u0 && isfinite(d.x)) x.x += (double)d.x * f0;
        if (u1 && isfinite(d.y)) x.y += (double)d.y * f1;
        p.Rp[idx] = x;
        p.RpS[idx] = df_split(x);
    }
}

// FP32 CG of one refinement round, Chronopoulos-Gear form, with no serial
// tail: the SpMV kernel adds its per-column sums to a double-buffered FP64
// accumulator with atomics, and every CTA of the following update kernel
// derives the same alpha, beta and convergence flags from them (identical
// inputs, identical arithmetic).  The CG state is double-buffered as well:
// update(it) reads slot it&1 and CTA 0 writes slot (it+1)&1.
//   inner32[0 .. 2P)        refinement state (skip, scale), written by k_refine_*
//   inner32[2P .. 4P)       CG state slot 0
//   inner32[4P .. 6P)       CG state slot 1
//   acc32[(slot*4 + q)*P + c]  gamma_re, gamma_im, delta_re, delta_im of column c

// Packed FP32 FMA of Blackwell (two lanes per instruction): d = a * b + c
// elementwise on float2.  The block products below broadcast one S entry
// into both lanes, so one instruction updates the real and imaginary parts
// of one complex column.
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) {
    unsigned long long ra, rb, rc, rd;
    asm("mov.b64 %0, {%1, %2};" : "=l"(ra) : "f"(a.x), "f"(a.y));
    asm("mov.b64 %0, {%1, %2};" : "=l"(rb) : "f"(b.x), "f"(b.y));
    asm("mov.b64 %0, {%1, %2};" : "=l"(rc) : "f"(c.x), "f"(c.y));
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(rd) : "l"(ra), "l"(rb), "l"(rc));
    float2 d;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(d.x), "=f"(d.y) : "l"(rd));
    return d;
}

// CG scalars of iteration it, once, by the last CTA of the SpMV to finish
// (every thread of that CTA calls this): FP64 alpha, beta and the
// convergence of every real column from the accumulated sums; the update
// kernel that follows only reads them (cgs[0..2P) alpha, [2P..4P) beta,
// upd flags in cgu[0..2P)).  The sums are read through L2 (__ldcg): other
// CTAs added them with device-scope atomics before their fence and ticket.
__device__ void inner32_scalars_cta(const PanelDev& p, int it) {
    __shared__ int s_cnt, s_err;
    const int P = p.P;
    const InnerState* base = p.inner32;
    const InnerState* prev = p.inner32 + (size_t)(1 + (it & 1)) * 2 * P;
    InnerState* next = p.inner32 + (size_t)(1 + ((it + 1) & 1)) * 2 * P;
    const double* acc_slot = p.acc32 + (size_t)(it & 1) * 4 * P;
    if (threadIdx.x == 0) { s_cnt = 0; s_err = 0; }
    __syncthreads();
    for (int rc = threadIdx.x; rc < 2 * P; rc += blockDim.x) {
        const int c = rc >> 1, part = rc & 1;
        const bool cact = p.col[c].active != 0;
        InnerState st = prev[rc];
        const double gam = __ldcg(acc_slot + (size_t)part * P + c);
        const double del = __ldcg(acc_slot + (size_t)(2 + part) * P + c);
        if (it == 0) {
            st.bnorm2 = gam;
            st.conv = (!cact || base[rc].skip || gam == 0.0) ? 1 : 0;
        }
        if (!st.conv) {
            if (gam <= p.inner_lo_tol * p.inner_lo_tol * st.bnorm2) {
                st.conv = 1;
            } else {
                const double beta = (it == 0) ? 0.0 : gam / st.gamma_prev;
                const double den = del - ((it == 0) ? 0.0 : beta * gam / st.alpha);
                // In exact arithmetic p^T S p >= r^T S r / cond(S); p^T S p <= 0 at
                // the first iteration (r^T S r <= 0), or while the residual is above
                // 1 % of its start, means S is not positive definite.  Otherwise a
                // non-positive or collapsed value is cancellation in the FP32
                // recurrences: the round stops and the FP64 refinement residual
                // decides what is left (counted in flags[5]).
                if (!(den > 0.0) || (it > 0 && den < 1e-4 * del)) {
                    if (it == 0 || (!(den > 0.0) && gam > 1e-4 * st.bnorm2)) s_err = 1;
                    else s_err = 2;
                    if (p.dbg) {
                        p.dbg[0] = it; p.dbg[1] = rc; p.dbg[2] = gam; p.dbg[3] = del;
                        p.dbg[4] = den; p.dbg[5] = st.bnorm2; p.dbg[6] = st.gamma_prev; p.dbg[7] = st.alpha;
                    }
                    st.conv = 1;
                } else {
                    st.alpha = gam / den;
                    st.beta = beta;
                    st.gamma_prev = gam;
                }
            }
        }
        p.cgs[rc] = st.alpha;
        p.cgs[2 * P + rc] = st.beta;
        p.cgu[rc] = st.conv ? 0 : 1;
        if (!st.conv) atomicAdd(&s_cnt, 1);
        next[rc] = st;
        if (p.hist && it < HIST_IT) {
            double* hh = p.hist + ((size_t)it * 2 * P + rc) * 4;
            hh[0] = gam; hh[1] = del; hh[2] = st.conv ? 0.0 : st.alpha; hh[3] = st.conv ? 0.0 : st.beta;
        }
    }
    double* acc_next = p.acc32 + (size_t)((it + 1) & 1) * 4 * P;
    for (int q = threadIdx.x; q < 4 * P; q += blockDim.x) acc_next[q] = 0.0;
    __syncthreads();
    if (threadIdx.x == 0) {
        p.flags[1] = s_cnt;
        if (s_cnt == 0) p.flags[3] = it;
        if (s_err == 1) atomicOr(&p.flags[0], ERR_NOT_SPD);
        if (s_err == 2) atomicAdd(&p.flags[5], 1);
        p.flags[7] = it;            // iteration whose scalars cgs/cgu hold
        *p.ticket32 = 0u;           // the next SpMV counts from zero
    }
}

// Completion ticket of the FP32 SpMV kernels: every CTA fences its atomic
// sums and takes a ticket; the CTA with the last one derives the CG scalars.
// No CTA waits for another.
__device__ void inner32_ticket_tail(const PanelDev& p, int it) {
    __shared__ bool s_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(p.ticket32, 1u) == gridDim.x - 1;
    __syncthreads();
    if (s_last) {
        __threadfence();
        inner32_scalars_cta(p, it);
    }
}

// w = S r (FP32) and the sums gamma = r.r, delta = w.r of every real column.
// CPT complex columns per thread (2: one float4 per orbital row), P / CPT
// threads per block row; the block-column index of the next block is loaded
// one block ahead so the panel-row gathers do not wait on it.
// PW: the panel width as a compile-time constant (4 ... 256: row strides
// fold into the load offsets; measured 4 % faster at 256 columns), 0 for
// any width at run time.
template <int CPT, int PW = 0>
__global__ void __launch_bounds__(THREADS, 4) k_inner32_spmv(DevSystem s, PanelDev p, int it) {
    __shared__ double smem[4 * CPT * THREADS];
    if (*(volatile int*)&p.flags[1] == 0) return;
    const int P = PW > 0 ? PW : p.P;
    const int TPR = P / CPT;                    // threads per block row
    const int t0 = threadIdx.x % TPR;
    const int c0 = t0 * CPT;
    const InnerState* base = p.inner32;
    const InnerState* cgp = p.inner32 + (size_t)(1 + (it & 1)) * 2 * P;
    bool live = false;
#pragma unroll
    for (int j = 0; j < CPT; ++j) {
        const int c = c0 + j;
        live |= p.col[c].active && (it == 0 ? !(base[2 * c].skip && base[2 * c + 1].skip)
                                            : !(cgp[2 * c].conv && cgp[2 * c + 1].conv));
    }
    float v32[4 * CPT];
#pragma unroll
    for (int q = 0; q < 4 * CPT; ++q) v32[q] = 0.f;
    const long long items = (long long)s.n_atoms * TPR;
    if (live) {
        for (long long idx = blockIdx.x * (long long)THREADS + threadIdx.x; idx < items;
             idx += (long long)gridDim.x * THREADS) {
            const int I = (int)(idx / TPR);
            float acc[4][2 * CPT];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int q = 0; q < 2 * CPT; ++q) acc[a][q] = 0.f;
            const int b0 = s.brow[I], b1 = s.brow[I + 1];
            int Jn = __ldg(s.bcol + b0);
            for (int bb = b0; bb < b1; ++bb) {
                const int J = Jn;
                if (bb + 1 < b1) Jn = __ldg(s.bcol + bb + 1);
                float xv[4][2 * CPT];
                const float2* xb = p.r32 + (size_t)(4 * J) * P + c0;
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const float2* xr = xb + e * P;
                    if (CPT == 2) {
                        const float4 q4 = *reinterpret_cast<const float4*>(xr);
                        xv[e][0] = q4.x; xv[e][1] = q4.y; xv[e][2] = q4.z; xv[e][3] = q4.w;
                    } else {
                        const float2 q2 = *xr;
                        xv[e][0] = q2.x; xv[e][1] = q2.y;
                    }
                }
                const float4* Sb = reinterpret_cast<const float4*>(s.S32 + 16 * (size_t)bb);
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    const float4 sr = __ldg(Sb + a);
#pragma unroll
                    for (int q = 0; q < 2 * CPT; ++q)
                        acc[a][q] += sr.x * xv[0][q] + sr.y * xv[1][q] + sr.z * xv[2][q] + sr.w * xv[3][q];
                }
            }
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                const size_t e = (size_t)(4 * I + a) * P + c0;
                float r[2 * CPT];
                if (CPT == 2) {
                    const float4 r4 = *reinterpret_cast<const float4*>(p.r32 + e);
                    r[0] = r4.x; r[1] = r4.y; r[2] = r4.z; r[3] = r4.w;
                    *reinterpret_cast<float4*>(p.w32 + e) = make_float4(acc[a][0], acc[a][1], acc[a][2], acc[a][3]);
                } else {
                    const float2 r2 = p.r32[e];
                    r[0] = r2.x; r[1] = r2.y;
                    p.w32[e] = make_float2(acc[a][0], acc[a][1]);
                }
#pragma unroll
                for (int j = 0; j < CPT; ++j) {
                    v32[4 * j + 0] += r[2 * j] * r[2 * j];
                    v32[4 * j + 1] += r[2 * j + 1] * r[2 * j + 1];
                    v32[4 * j + 2] += acc[a][2 * j] * r[2 * j];
                    v32[4 * j + 3] += acc[a][2 * j + 1] * r[2 * j + 1];
                }
            }
        }
    }
    double v[4 * CPT];
#pragma unroll
    for (int q = 0; q < 4 * CPT; ++q) v[q] = v32[q];
    block_reduce_cols<4 * CPT>(v, TPR, smem);
    if (threadIdx.x < TPR) {
        double* acc_slot = p.acc32 + (size_t)(it & 1) * 4 * P;
#pragma unroll
        for (int j = 0; j < CPT; ++j) {
            const int c = threadIdx.x * CPT + j;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const double val = smem[(4 * j + q) * THREADS + threadIdx.x];
                if (val != 0.0) atomicAdd(acc_slot + (size_t)q * P + c, val);
            }
        }
    }
    inner32_ticket_tail(p, it);
}

__device__ __forceinline__ uint32_t smem_u32(const void* ptr) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(ptr));
}

// Grouped form: CTA (g, slice) computes the 4G rows of the G consecutive
// atoms of group g for the PC complex columns of one panel slice.  The panel
// rows of the distinct block columns of the group (its neighbour union, built
// on the host when the system is created) and the group's FP32 S blocks are
// staged once in shared memory by 16-byte asynchronous copies; every block
// product then reads shared memory.  The union of 16 neighbouring atoms is
// ~3x smaller than the sum of their neighbour lists, so the L2 -> SM gather
// traffic drops by that factor.  PC / 2 threads per atom, two complex
// columns each; the block products pair (S[a][e], S[a][e+1]), two adjacent
// lanes of a loaded S row, against (x[e][q], x[e+1][q]) in packed FP32 FMAs.
constexpr int PC = 32;
constexpr int GRP_HDR = 128;   // reserved head of the dynamic shared memory

__global__ void __launch_bounds__(256) k_inner32_spmv_grp(DevSystem s, PanelDev p, int it) {
    extern __shared__ __align__(128) unsigned char gsm[];
    if (*(volatile int*)&p.flags[1] == 0) return;
    const int P = p.P;
    const int nslices = P / PC;
    const int g = blockIdx.x / nslices;
    const int slice = blockIdx.x - g * nslices;
    const int a0 = g * s.grpG;
    const int a1 = min(a0 + s.grpG, s.n_atoms);
    const int u0 = s.grp_ptr[g];
    const int U = s.grp_ptr[g + 1] - u0;
    const int bb0 = s.brow[a0];
    const int nbk = s.brow[a1] - bb0;
    constexpr int TPA = PC / 2;
    const int t = threadIdx.x;
    const int I = a0 + t / TPA;
    const int tc = t % TPA;
    const int c0 = slice * PC + 2 * tc;
    const InnerState* base = p.inner32;
    const InnerState* cgp = p.inner32 + (size_t)(1 + (it & 1)) * 2 * P;
    bool live = false;
    if (I < a1) {
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int c = c0 + j;
            live |= p.col[c].active && (it == 0 ? !(base[2 * c].skip && base[2 * c + 1].skip)
                                                : !(cgp[2 * c].conv && cgp[2 * c + 1].conv));
        }
    }
    const bool any_live = __syncthreads_or(live);
    const size_t xregion = (size_t)s.max_union * 4 * PC * sizeof(float2);
    const size_t red_bytes = (size_t)(blockDim.x / 32) * TPA * 8 * sizeof(double);
    float4* xs = reinterpret_cast<float4*>(gsm + GRP_HDR);                       // [U][4][PC/2]
    double* red = reinterpret_cast<double*>(gsm + GRP_HDR);                      // aliases xs after use
    const float4* ss = reinterpret_cast<const float4*>(gsm + GRP_HDR + (xregion > red_bytes ? xregion : red_bytes));
    // stage the union's panel rows (16 float4 per row of the slice) and the
    // group's S blocks with 16-byte asynchronous copies by every thread
    if (any_live) {
        const int nx = U * 4 * TPA;               // float4 of the union rows
        const uint32_t xs_a = smem_u32(xs);
        for (int k = t; k < nx; k += blockDim.x) {
            const int row = k / TPA, q4 = k - row * TPA;
            const int J = __ldg(s.grp_cols + u0 + row / 4);
            const float2* src = p.r32 + (size_t)(4 * J + (row & 3)) * P + slice * PC + 2 * q4;
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(xs_a + 16u * (uint32_t)k), "l"(src));
        }
        const uint32_t ss_a = smem_u32(ss);
        const float4* sg = reinterpret_cast<const float4*>(s.S32 + 16 * (size_t)bb0);
        for (int k = t; k < nbk * 4; k += blockDim.x)
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(ss_a + 16u * (uint32_t)k), "l"(sg + k));
        asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;" ::: "memory");
    }
    __syncthreads();
    float v32[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) v32[q] = 0.f;
    if (live) {
        float2 acc2[4][4];   // (even e, odd e) partial sums of row a, value q
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc2[a][q] = make_float2(0.f, 0.f);
        const int b0 = s.brow[I], b1 = s.brow[I + 1];
        int jn = __ldg(s.blk_loc + b0);
        for (int bb = b0; bb < b1; ++bb) {
            const int j = jn;
            if (bb + 1 < b1) jn = __ldg(s.blk_loc + bb + 1);
            const float4* xj = xs + (size_t)j * 4 * TPA + tc;
            float xv[4][4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const float4 q4 = xj[e * TPA];
                xv[e][0] = q4.x; xv[e][1] = q4.y; xv[e][2] = q4.z; xv[e][3] = q4.w;
            }
            float2 xp[2][4];
#pragma unroll
            for (int h = 0; h < 2; ++h)
#pragma unroll
                for (int q = 0; q < 4; ++q) xp[h][q] = make_float2(xv[2 * h][q], xv[2 * h + 1][q]);
            const float4* Sb = ss + (size_t)(bb - bb0) * 4;
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                const float4 sr = Sb[a];
                const float2 s01 = make_float2(sr.x, sr.y), s23 = make_float2(sr.z, sr.w);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    acc2[a][q] = ffma2(s01, xp[0][q], acc2[a][q]);
                    acc2[a][q] = ffma2(s23, xp[1][q], acc2[a][q]);
                }
            }
        }
        float acc[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[a][q] = acc2[a][q].x + acc2[a][q].y;
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            const size_t e = (size_t)(4 * I + a) * P + c0;
            const float4 r4 = *reinterpret_cast<const float4*>(p.r32 + e);
            *reinterpret_cast<float4*>(p.w32 + e) = make_float4(acc[a][0], acc[a][1], acc[a][2], acc[a][3]);
            const float r[4] = {r4.x, r4.y, r4.z, r4.w};
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                v32[4 * j + 0] += r[2 * j] * r[2 * j];
                v32[4 * j + 1] += r[2 * j + 1] * r[2 * j + 1];
                v32[4 * j + 2] += acc[a][2 * j] * r[2 * j];
                v32[4 * j + 3] += acc[a][2 * j + 1] * r[2 * j + 1];
            }
        }
    }
    // sums over the atoms of the CTA: the two atoms of a warp by shuffle, the
    // warps through shared memory, then one atomic per column and sum
    double v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) v[q] = (double)v32[q] + __shfl_xor_sync(0xffffffffu, (double)v32[q], TPA);
    __syncthreads();   // all reads of the staged panel rows are done; red aliases them
    const int warp = t / 32, lane = t % 32;
    if (lane < TPA)
#pragma unroll
        for (int q = 0; q < 8; ++q) red[((size_t)warp * TPA + lane) * 8 + q] = v[q];
    __syncthreads();
    for (int k = t; k < TPA * 8; k += blockDim.x) {
        const int tcol = k % TPA, q = k / TPA;      // q = 4 * j + component
        double sum = 0.0;
        for (int w = 0; w < (int)(blockDim.x / 32); ++w) sum += red[((size_t)w * TPA + tcol) * 8 + q];
        const int c = slice * PC + 2 * tcol + q / 4;
        if (sum != 0.0) atomicAdd(p.acc32 + (size_t)(it & 1) * 4 * P + (size_t)(q % 4) * P + c, sum);
    }
    inner32_ticket_tail(p, it);
}


// p = r + beta p, s = w + beta s, x += alpha p, r -= alpha s (FP32) with the
// scalars that the last CTA of the SpMV derived.  At it == 0 every vector
// is initialised.
template <int V>
__global__ void k_inner32_update(PanelDev p, int it) {
    // V complex columns per thread (V = 2: one float4 of each vector)
    using vec = typename std::conditional<V == 2, float4, float2>::type;
    const int P = p.P;
    if (*(volatile int*)&p.flags[7] != it) return;      // no scalars for this iteration (the SpMV exited early)
    const int c0 = (V * threadIdx.x) % P;
    // per real column q: act (the complex column is active: at it == 0 its
    // p, s, x start at zero) and upd (this iteration updates it); inactive
    // columns keep their vectors
    float a[2 * V], b[2 * V];
    bool act[2 * V], upd[2 * V];
    bool any = false;
#pragma unroll
    for (int j = 0; j < V; ++j) {
        const int c = c0 + j;
        const bool ac = p.col[c].active != 0;
#pragma unroll
        for (int part = 0; part < 2; ++part) {
            const int q = 2 * j + part, rc = 2 * c + part;
            act[q] = ac;
            upd[q] = ac && p.cgu[rc] != 0;
            a[q] = upd[q] ? (float)p.cgs[rc] : 0.f;
            b[q] = upd[q] ? (float)p.cgs[2 * P + rc] : 0.f;
            any |= (it == 0) ? act[q] : upd[q];
        }
    }
    if (!any) return;
    const long long items = (long long)p.npad * P / V;
    vec* r32 = reinterpret_cast<vec*>(p.r32);
    vec* w32 = reinterpret_cast<vec*>(p.w32);
    vec* p32 = reinterpret_cast<vec*>(p.p32);
    vec* s32 = reinterpret_cast<vec*>(p.s32);
    vec* x32 = reinterpret_cast<vec*>(p.x32);
    for (long long idx = blockIdx.x * (long long)THREADS + threadIdx.x; idx < items;
         idx += (long long)gridDim.x * THREADS) {
        const vec rv = r32[idx], wv = w32[idx];
        vec pv = p32[idx], sv = s32[idx], xv = x32[idx];
        vec rn = rv;
        const float* r = reinterpret_cast<const float*>(&rv);
        const float* w = reinterpret_cast<const float*>(&wv);
        float* pp = reinterpret_cast<float*>(&pv);
        float* ss = reinterpret_cast<float*>(&sv);
        float* xx = reinterpret_cast<float*>(&xv);
        float* rr = reinterpret_cast<float*>(&rn);
#pragma unroll
        for (int q = 0; q < 2 * V; ++q) {
            if (it == 0 && act[q]) {
                pp[q] = 0.f;
                ss[q] = 0.f;
                xx[q] = 0.f;
            }
            if (upd[q]) {
                pp[q] = r[q] + b[q] * pp[q];
                ss[q] = w[q] + b[q] * ss[q];
                xx[q] += a[q] * pp[q];
                rr[q] = r[q] - a[q] * ss[q];
            }
        }
        p32[idx] = pv;
        s32[idx] = sv;
        x32[idx] = xv;
        r32[idx] = rn;
    }
}

// ---------------------------------------------------------------------------
// FP32 corrections of a refinement round by Chebyshev iteration (the default
// of TB_MIXED).  With the spectrum of S inside [a, b] (bounds from a Lanczos
// run on S, with margins), gamma = 2 / (a + b) and sigma = (b - a) / (b + a),
// the semi-iterative recurrence
//     d_0 = 0,  d_1 = gamma f,
//     d_{k+1} = d_{k-1} + omega_{k+1} (gamma (f - S d_k) + d_k - d_{k-1}),
//     omega_2 = 1 / (1 - sigma^2 / 2),  omega_{k+1} = 1 / (1 - omega_k sigma^2 / 4),
// reduces the error of S d = f by 1 / T_k(1 / sigma) after k steps (T_k the
// Chebyshev polynomial).  Its coefficients are fixed in advance, so a step
// needs no inner product: the product S d_k and the update of the own rows
// are one kernel, and the FP64 residual of the refinement decides what is
// left.  d_k and d_{k-1} alternate between x32 and p32; d_{k+1} overwrites
// d_{k-1} in place (each element is read and written by one thread only,
// and the gather reads d_k alone).  f is the round's right-hand side r32.
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool cheb_live(const PanelDev& p, int c) {
    return p.col[c].active && !(p.inner32[2 * c].skip && p.inner32[2 * c + 1].skip);
}

// One Chebyshev step: io <- io + omega (gamma (f - S cur) + cur - io) on the
// own rows, with S cur gathered as in k_inner32_spmv (CPT complex columns
// per thread, P / CPT threads per block row, PW the panel width when it is
// a compile-time constant).  mode 1: the first step (d_0 = 0, io is not
// read).  mode 2 (the LAST instance): the last step, which adds its result
// to the FP64 solution of the refinement instead of storing it
// (x += d_n / scale and the double-float split, as k_refine_add; a
// non-finite value is dropped).  When every diagonal block of S is the
// identity (s.unit_diag: orthonormal orbitals on one atom), the gather skips
// it and S cur = (S - 1) cur + cur takes the own rows of cur, which the
// update reads anyway: one block of ~17 per block row fewer to gather.
template <int CPT, int PW = 0, bool LAST = false>
__global__ void __launch_bounds__(THREADS, 4) k_inner32_cheb(DevSystem s, PanelDev p, const float2* __restrict__ cur,
                                                            float2* io, float omega, float gamma, int mode) {
    if (*(volatile int*)&p.flags[4] == 0) return;
    const int P = PW > 0 ? PW : p.P;
    const int TPR = P / CPT;
    const int t0 = threadIdx.x % TPR;
    const int c0 = t0 * CPT;
    bool live = false;
#pragma unroll
    for (int j = 0; j < CPT; ++j) live |= cheb_live(p, c0 + j);
    if (!live) return;
    const long long items = (long long)s.n_atoms * TPR;
    for (long long idx = blockIdx.x * (long long)THREADS + threadIdx.x; idx < items;
         idx += (long long)gridDim.x * THREADS) {
        const int I = (int)(idx / TPR);
        float acc[4][2 * CPT];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int q = 0; q < 2 * CPT; ++q) acc[a][q] = 0.f;
        const int b0 = s.brow[I], b1 = s.brow[I + 1];
        int Jn = __ldg(s.bcol + b0);
        for (int bb = b0; bb < b1; ++bb) {
            const int J = Jn;
            if (bb + 1 < b1) Jn = __ldg(s.bcol + bb + 1);
            if (s.unit_diag && J == I) continue;   // S_II = 1: d_I is added in the update
            float xv[4][2 * CPT];
            const float2* xb = cur + (size_t)(4 * J) * P + c0;
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const float2* xr = xb + e * P;
                if (CPT == 2) {
                    const float4 q4 = *reinterpret_cast<const float4*>(xr);
                    xv[e][0] = q4.x; xv[e][1] = q4.y; xv[e][2] = q4.z; xv[e][3] = q4.w;
                } else {
                    const float2 q2 = *xr;
                    xv[e][0] = q2.x; xv[e][1] = q2.y;
                }
            }
            const float4* Sb = reinterpret_cast<const float4*>(s.S32 + 16 * (size_t)bb);
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                const float4 sr = __ldg(Sb + a);
#pragma unroll
                for (int q = 0; q < 2 * CPT; ++q)
                    acc[a][q] += sr.x * xv[0][q] + sr.y * xv[1][q] + sr.z * xv[2][q] + sr.w * xv[3][q];
            }
        }
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            const size_t e = (size_t)(4 * I + a) * P + c0;
            float f[2 * CPT], dc[2 * CPT], dp[2 * CPT];
            if (CPT == 2) {
                const float4 f4 = *reinterpret_cast<const float4*>(p.r32 + e);
                const float4 c4 = *reinterpret_cast<const float4*>(cur + e);
                const float4 p4 = mode == 1 ? make_float4(0.f, 0.f, 0.f, 0.f) : *reinterpret_cast<const float4*>(io + e);
                f[0] = f4.x; f[1] = f4.y; f[2] = f4.z; f[3] = f4.w;
                dc[0] = c4.x; dc[1] = c4.y; dc[2] = c4.z; dc[3] = c4.w;
                dp[0] = p4.x; dp[1] = p4.y; dp[2] = p4.z; dp[3] = p4.w;
            } else {
                const float2 f2 = p.r32[e], c2 = cur[e], p2 = mode == 1 ? make_float2(0.f, 0.f) : io[e];
                f[0] = f2.x; f[1] = f2.y; dc[0] = c2.x; dc[1] = c2.y; dp[0] = p2.x; dp[1] = p2.y;
            }
            float dn[2 * CPT];
#pragma unroll
            for (int q = 0; q < 2 * CPT; ++q) dn[q] = dp[q] + omega * (gamma * (f[q] - (s.unit_diag ? acc[a][q] + dc[q] : acc[a][q])) + dc[q] - dp[q]);
            if (LAST) {
#pragma unroll
                for (int j = 0; j < CPT; ++j) {
                    // 1 / scale of the real columns that took the round (0: skipped)
                    const InnerState i0 = p.inner32[2 * (c0 + j)], i1 = p.inner32[2 * (c0 + j) + 1];
                    const bool ca = p.col[c0 + j].active != 0;
                    double2 x = p.Rp[e + j];
                    if (ca && !i0.skip && isfinite(dn[2 * j])) x.x += (double)dn[2 * j] * i0.unscale;
                    if (ca && !i1.skip && isfinite(dn[2 * j + 1])) x.y += (double)dn[2 * j + 1] * i1.unscale;
                    p.Rp[e + j] = x;
                    p.RpS[e + j] = df_split(x);
                }
            } else if (CPT == 2) {
                *reinterpret_cast<float4*>(io + e) = make_float4(dn[0], dn[1], dn[2], dn[3]);
            } else {
                io[e] = make_float2(dn[0], dn[1]);
            }
        }
    }
}

// The same Chebyshev step with four complex columns per thread and packed
// FP32 FMAs: thread t0 of a block row (P / 4 threads per row) takes the
// column pairs (2 t0, 2 t0 + 1) and (P/2 + 2 t0, P/2 + 2 t0 + 1), so each of
// its two loads per gathered row is part of a contiguous 512-byte warp
// access.  The block product runs over the rows e of the gathered d_k: row e
// of the transposed block (column e of S_IJ, from S32T) gives S[a][e] for
// the four output rows a, each broadcast into both lanes of a packed FMA
// against the (re, im) pairs of the thread's columns.  Against two columns
// per thread this halves the S loads and the FMA instructions per column
// (ncu at P = 128: 7.3 M instead of 15.5 M warp instructions per launch).
// Compiled for three CTAs per SM (80 registers): at four (64 registers) the
// 32 accumulators spill.  Measured on the benchmark workload, four panels in
// flight: 17.2 M shift*RHS*iterations/s against 15.8 M with two columns per
// thread; eight columns per thread (two CTAs per SM), staging the next
// block's rows in shared memory, and L1 / L2 prefetches of them all measured
// slower.
__device__ __forceinline__ float2 lo2(float4 v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(float4 v) { return make_float2(v.z, v.w); }

template <int PW, bool LAST>
__global__ void __launch_bounds__(THREADS, 3) k_inner32_cheb4(DevSystem s, PanelDev p, const float2* __restrict__ cur,
                                                             float2* io, float omega, float gamma, int mode) {
    constexpr int CPT = 4, NP = 2;   // columns, column pairs per thread
    if (*(volatile int*)&p.flags[4] == 0) return;
    const int P = PW > 0 ? PW : p.P;
    const int TPR = P / CPT;
    const int pstride = P / NP;
    const int t0 = threadIdx.x % TPR;
    bool live = false;
#pragma unroll
    for (int k = 0; k < NP; ++k) live |= cheb_live(p, k * pstride + 2 * t0) || cheb_live(p, k * pstride + 2 * t0 + 1);
    if (!live) return;
    const long long items = (long long)s.n_atoms * TPR;
    for (long long idx = blockIdx.x * (long long)THREADS + threadIdx.x; idx < items;
         idx += (long long)gridDim.x * THREADS) {
        const int I = (int)(idx / TPR);
        float2 acc[4][CPT];   // [output row a][column 2k, 2k + 1 of pair k] (re, im)
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int q = 0; q < CPT; ++q) acc[a][q] = make_float2(0.f, 0.f);
        const int b0 = s.brow[I], b1 = s.brow[I + 1];
        int Jn = __ldg(s.bcol + b0);
        for (int bb = b0; bb < b1; ++bb) {
            const int J = Jn;
            if (bb + 1 < b1) Jn = __ldg(s.bcol + bb + 1);
            if (s.unit_diag && J == I) continue;   // S_II = 1: d_I is added in the update
            const float2* xb = cur + (size_t)(4 * J) * P + 2 * t0;
            const float4* St = reinterpret_cast<const float4*>(s.S32T + 16 * (size_t)bb);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                float4 xq[NP];
#pragma unroll
                for (int k = 0; k < NP; ++k) xq[k] = *reinterpret_cast<const float4*>(xb + (size_t)e * P + k * pstride);
                const float4 sc = __ldg(St + e);     // S[0][e], S[1][e], S[2][e], S[3][e]
                const float sv[4] = {sc.x, sc.y, sc.z, sc.w};
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    const float2 s2 = make_float2(sv[a], sv[a]);
#pragma unroll
                    for (int k = 0; k < NP; ++k) {
                        acc[a][2 * k] = __ffma2_rn(s2, lo2(xq[k]), acc[a][2 * k]);
                        acc[a][2 * k + 1] = __ffma2_rn(s2, hi2(xq[k]), acc[a][2 * k + 1]);
                    }
                }
            }
        }
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            const size_t row = (size_t)(4 * I + a) * P;
#pragma unroll
            for (int k = 0; k < NP; ++k) {
                const int c = k * pstride + 2 * t0;
                const size_t e = row + c;
                const float4 f4 = *reinterpret_cast<const float4*>(p.r32 + e);
                const float4 c4 = *reinterpret_cast<const float4*>(cur + e);
                const float4 p4 = mode == 1 ? make_float4(0.f, 0.f, 0.f, 0.f) : *reinterpret_cast<const float4*>(io + e);
                const float2 y0 = acc[a][2 * k], y1 = acc[a][2 * k + 1];
                const float f[4] = {f4.x, f4.y, f4.z, f4.w}, dc[4] = {c4.x, c4.y, c4.z, c4.w};
                const float dp[4] = {p4.x, p4.y, p4.z, p4.w}, y[4] = {y0.x, y0.y, y1.x, y1.y};
                float dn[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) dn[q] = dp[q] + omega * (gamma * (f[q] - (s.unit_diag ? y[q] + dc[q] : y[q])) + dc[q] - dp[q]);
                if (LAST) {
#pragma unroll
                    for (int j = 0; j < 2; ++j) {
                        const InnerState i0 = p.inner32[2 * (c + j)], i1 = p.inner32[2 * (c + j) + 1];
                        const bool ca = p.col[c + j].active != 0;
                        double2 x = p.Rp[e + j];
                        if (ca && !i0.skip && isfinite(dn[2 * j])) x.x += (double)dn[2 * j] * i0.unscale;
                        if (ca && !i1.skip && isfinite(dn[2 * j + 1])) x.y += (double)dn[2 * j + 1] * i1.unscale;
                        p.Rp[e + j] = x;
                        p.RpS[e + j] = df_split(x);
                    }
                } else {
                    *reinterpret_cast<float4*>(io + e) = make_float4(dn[0], dn[1], dn[2], dn[3]);
                }
            }
        }
    }
}

// The four-column Chebyshev step for systems with s-only atoms (water: O
// with s, p and H with s): block rows in the order of s.row_order (sp atoms,
// then s atoms), and every product with the real entries only -- an s atom
// J contributes one gathered row (not four), an s row atom I one output row
// -- read from the compact blocks.  The padded slots of the vectors are
// neither read nor written (the other kernels keep them at zero).
template <int PW, bool LAST>
__global__ void __launch_bounds__(THREADS, 3) k_inner32_cheb4r(DevSystem s, PanelDev p, const float2* __restrict__ cur,
                                                              float2* io, float omega, float gamma, int mode) {
    constexpr int NP = 2;
    if (*(volatile int*)&p.flags[4] == 0) return;
    const int P = PW > 0 ? PW : p.P;
    const int TPR = P / 4;
    const int pstride = P / NP;
    const int t0 = threadIdx.x % TPR;
    bool live = false;
#pragma unroll
    for (int k = 0; k < NP; ++k) live |= cheb_live(p, k * pstride + 2 * t0) || cheb_live(p, k * pstride + 2 * t0 + 1);
    if (!live) return;
    const long long items = (long long)s.n_atoms * TPR;
    for (long long idx = blockIdx.x * (long long)THREADS + threadIdx.x; idx < items;
         idx += (long long)gridDim.x * THREADS) {
        const int I = s.row_order[idx / TPR];
        const int ni = s.norb[I];
        float2 acc[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[a][q] = make_float2(0.f, 0.f);
        const int b0 = s.brow[I], b1 = s.brow[I + 1];
        // block metadata (column atom, compact offset, its orbital count)
        // one block ahead, so the gathers of a block wait on nothing else
        int2 mn = __ldg(s.bmeta + b0);
        for (int bb = b0; bb < b1; ++bb) {
            const int2 m = mn;
            if (bb + 1 < b1) mn = __ldg(s.bmeta + bb + 1);
            const int J = m.x;
            const int nj = (m.y < 0) ? 1 : 4;
            if (s.unit_diag && J == I) continue;   // S_II = 1: d_I is added in the update
            const float2* xb = cur + (size_t)(4 * J) * P + 2 * t0;
            const float4* Sr = reinterpret_cast<const float4*>(s.S32r) + (m.y & 0x7fffffff);
            if (ni == 4) {
                // nj rows e of the gathered d_k, column e of the block as four
                // rows a (unrolled with the row count as a predicate, so the
                // loads of all rows are issued together)
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    if (e >= nj) break;
                    const float4 xa = *reinterpret_cast<const float4*>(xb + (size_t)e * P);
                    const float4 xq = *reinterpret_cast<const float4*>(xb + (size_t)e * P + pstride);
                    const float4 sc = __ldg(Sr + e);
                    const float sv[4] = {sc.x, sc.y, sc.z, sc.w};
#pragma unroll
                    for (int a = 0; a < 4; ++a) {
                        const float2 s2 = make_float2(sv[a], sv[a]);
                        acc[a][0] = __ffma2_rn(s2, lo2(xa), acc[a][0]);
                        acc[a][1] = __ffma2_rn(s2, hi2(xa), acc[a][1]);
                        acc[a][2] = __ffma2_rn(s2, lo2(xq), acc[a][2]);
                        acc[a][3] = __ffma2_rn(s2, hi2(xq), acc[a][3]);
                    }
                }
            } else {
                // one output row: row 0 of the block (S[0][0 .. nj))
                const float4 sr = __ldg(Sr);
                const float sv[4] = {sr.x, sr.y, sr.z, sr.w};
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    if (e >= nj) break;
                    const float4 xa = *reinterpret_cast<const float4*>(xb + (size_t)e * P);
                    const float4 xq = *reinterpret_cast<const float4*>(xb + (size_t)e * P + pstride);
                    const float2 s2 = make_float2(sv[e], sv[e]);
                    acc[0][0] = __ffma2_rn(s2, lo2(xa), acc[0][0]);
                    acc[0][1] = __ffma2_rn(s2, hi2(xa), acc[0][1]);
                    acc[0][2] = __ffma2_rn(s2, lo2(xq), acc[0][2]);
                    acc[0][3] = __ffma2_rn(s2, hi2(xq), acc[0][3]);
                }
            }
        }
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            if (a >= ni) break;
            const size_t row = (size_t)(4 * I + a) * P;
#pragma unroll
            for (int k = 0; k < NP; ++k) {
                const int c = k * pstride + 2 * t0;
                const size_t e = row + c;
                const float4 f4 = *reinterpret_cast<const float4*>(p.r32 + e);
                const float4 c4 = *reinterpret_cast<const float4*>(cur + e);
                const float4 p4 = mode == 1 ? make_float4(0.f, 0.f, 0.f, 0.f) : *reinterpret_cast<const float4*>(io + e);
                const float2 y0 = acc[a][2 * k], y1 = acc[a][2 * k + 1];
                const float f[4] = {f4.x, f4.y, f4.z, f4.w}, dc[4] = {c4.x, c4.y, c4.z, c4.w};
                const float dp[4] = {p4.x, p4.y, p4.z, p4.w}, y[4] = {y0.x, y0.y, y1.x, y1.y};
                float dn[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) dn[q] = dp[q] + omega * (gamma * (f[q] - (s.unit_diag ? y[q] + dc[q] : y[q])) + dc[q] - dp[q]);
                if (LAST) {
#pragma unroll
                    for (int j = 0; j < 2; ++j) {
                        const InnerState i0 = p.inner32[2 * (c + j)], i1 = p.inner32[2 * (c + j) + 1];
                        const bool ca = p.col[c + j].active != 0;
                        double2 x = p.Rp[e + j];
                        if (ca && !i0.skip && isfinite(dn[2 * j])) x.x += (double)dn[2 * j] * i0.unscale;
                        if (ca && !i1.skip && isfinite(dn[2 * j + 1])) x.y += (double)dn[2 * j + 1] * i1.unscale;
                        p.Rp[e + j] = x;
                        p.RpS[e + j] = df_split(x);
                    }
                } else {
                    *reinterpret_cast<float4*>(io + e) = make_float4(dn[0], dn[1], dn[2], dn[3]);
                }
            }
        }
    }
}

// rho_{n+1} = r_{n+1}^T r'_{n+1} (unconjugated); also clears the count of
// active columns that the shift step rebuilds.
__global__ void __launch_bounds__(THREADS) k_finish(PanelDev p) {
    __shared__ double smem[2 * THREADS];
    const int P = p.P;
    const int c = threadIdx.x % P;
    double v[2] = {0.0, 0.0};
    if (p.col[c].active) {
        const long long items = (long long)p.npad * P;
        for (long long idx = blockIdx.x * (long long)THREADS + threadIdx.x; idx < items;
             idx += (long long)gridDim.x * THREADS) {
            const double2 m = cmul(p.Rcur[idx], p.Rp[idx]);
            v[0] += m.x;
            v[1] += m.y;
        }
    }
    if (grid_reduce_cols<2>(v, P, p, smem)) {
        const int t = threadIdx.x;
        if (t < P && p.col[t].active) p.col[t].rho_new = cmk(smem[t], smem[THREADS + t]);
        if (t == 0) p.flags[2] = 0;
    }
}

// Projected functionals f_m^T r' of column c into d[0..nfun).
__device__ void eval_functionals(const DevSystem& s, const PanelDev& p, int c, int nfun, double2* d,
                                 double* red) {
    const int tid = threadIdx.x;
    if (p.proj == PROJ_ROWS) {
        for (int m = tid; m < nfun; m += THREADS) d[m] = p.Rp[(size_t)p.frow[(size_t)c * p.M + m] * p.P + c];
    } else if (p.proj == PROJ_SROW) {
        // s_j^T r' = sum over row j of S (S symmetric)
        const int row = p.col[c].row, I = row >> 2, a = row & 3;
        const int b0 = s.brow[I], nbl = s.brow[I + 1] - b0;
        double re = 0.0, im = 0.0;
        for (int e = tid; e < 4 * nbl; e += THREADS) {
            const int b = b0 + e / 4, be = e % 4;
            const double sv = s.S[16 * (size_t)b + 4 * a + be];
            const double2 x = p.Rp[(size_t)(4 * s.bcol[b] + be) * p.P + c];
            re += sv * x.x;
            im += sv * x.y;
        }
        red[tid] = re;
        red[THREADS + tid] = im;
        __syncthreads();
        for (int st = THREADS / 2; st >= 1; st >>= 1) {
            if (tid < st) {
                red[tid] += red[tid + st];
                red[THREADS + tid] += red[THREADS + tid + st];
            }
            __syncthreads();
        }
        if (tid == 0) d[0] = cmk(red[0], red[THREADS]);
    }
    __syncthreads();
}

// Initial shift state: pi_0 = pi_{-1} = 1, x^k_0 = 0, p^k_0 = r'_0 (projected:
// u^k = f^T r'_0), rho_0 = r_0^T r'_0.
__global__ void k_shift_init(DevSystem s, PanelDev p) {
    extern __shared__ double2 dyn[];
    __shared__ double red[2 * THREADS];
    const int c = blockIdx.x, K = p.K;
    ColState cs = p.col[c];
    if (!cs.active) return;
    const int nfun = cs.nfun;
    double2* d = dyn;
    if (p.proj != PROJ_NONE) eval_functionals(s, p, c, nfun, d, red);
    for (int k = threadIdx.x; k < K; k += THREADS) {
        p.pi[(size_t)c * K + k] = cmk(1.0, 0.0);
        p.pi_prev[(size_t)c * K + k] = cmk(1.0, 0.0);
        p.conv_iter[(size_t)c * K + k] = -1;
    }
    if (p.proj != PROJ_NONE) {
        for (int e = threadIdx.x; e < K * nfun; e += THREADS) {
            const int k = e / nfun, m = e % nfun;
            const size_t o = ((size_t)c * K + k) * p.M + m;
            p.t[o] = cmk(0.0, 0.0);
            p.u[o] = d[m];
            if (p.deriv) {
                p.dt[o] = cmk(0.0, 0.0);
                p.du[o] = cmk(0.0, 0.0);      // u_0 = F r'_0 does not depend on z_k
            }
        }
    }
    if (p.deriv)
        for (int k = threadIdx.x; k < K; k += THREADS) {
            p.dpi[(size_t)c * K + k] = cmk(0.0, 0.0);
            p.dpi_prev[(size_t)c * K + k] = cmk(0.0, 0.0);
        }
    __syncthreads();
    if (threadIdx.x == 0) {
        cs.rho = cs.rho_new;
        cs.n_unconv = K;
        p.col[c] = cs;
        atomicAdd(&p.flags[2], 1);
    }
}

__global__ void k_full_init(PanelDev p) {
    const long long per = (long long)p.npad * p.P;
    const long long items = per * p.K;
    for (long long idx = blockIdx.x * (long long)THREADS + threadIdx.x; idx < items;
         idx += (long long)gridDim.x * THREADS) {
        p.X[idx] = cmk(0.0, 0.0);
        p.Pk[idx] = p.Rp[idx % per];
    }
}

// ---------------------------------------------------------------------------
// a5 + a6: every shift of column c in one pass (Eq. shift:pi, Eq. collinear),
// projected updates, convergence, and seed switching on the device.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(THREADS) k_shift_step(DevSystem s, PanelDev p) {
    extern __shared__ double2 dyn[];
    __shared__ double red[2 * THREADS];
    __shared__ int s_cnt[THREADS];
    __shared__ double s_best[THREADS];
    __shared__ int s_bestk[THREADS];
    __shared__ int s_sw;
    __shared__ double2 s_c1, s_c0;
    const int c = blockIdx.x, K = p.K, tid = threadIdx.x;
    const ColState cs = p.col[c];
    if (!cs.active) {
        if (p.proj == PROJ_NONE)
            for (int k = tid; k < K; k += THREADS) p.ipi[(size_t)c * K + k] = cmk(0.0, 0.0);
        return;
    }
    const int nfun = cs.nfun;
    double2* d = dyn;                       // [M]
    double2* sak = d + p.M;                 // [K]
    double2* sbk = sak + K;                 // [K]
    double2* sip = sbk + K;                 // [K]
    double2* sdak = sip + K;                // [K] derivative mode: d alpha^k, d beta^k, d (1/pi^k)
    double2* sdbk = sdak + K;
    double2* sdip = sdbk + K;
    if (p.proj != PROJ_NONE) eval_functionals(s, p, c, nfun, d, red);

    const double2 one = cmk(1.0, 0.0);
    const double2 alpha = cs.alpha;
    const double2 beta = cdiv(cs.rho_new, cs.rho);
    const double2 c2 = cdiv(cmul(cs.beta_prev, alpha), cs.alpha_prev);
    const double rnorm = cs.rnorm;
    const int it = cs.iters;
    int nunc = 0;
    double best = -1.0;
    int bestk = K;
    for (int k = tid; k < K; k += THREADS) {
        const size_t o = (size_t)c * K + k;
        if (p.conv_iter[o] >= 0) {
            sip[k] = cmk(0.0, 0.0);
            if (p.proj == PROJ_NONE) p.ipi[o] = cmk(0.0, 0.0);
            continue;
        }
        const double2 pk = p.pi[o], pp = p.pi_prev[o];
        const double2 dl = csub(p.z[k], cs.zs);
        const double2 pin = cadd(cmul(cadd(one, cmul(alpha, dl)), pk), cmul(c2, csub(pk, pp)));
        const double2 ratio = cdiv(pk, pin);
        const double2 ak = cmul(alpha, ratio);
        const double2 bk = cmul(beta, cmul(ratio, ratio));
        const double2 ip = cdiv(one, pin);
        const double res = rnorm / cabs2(pin);
        p.pi_prev[o] = pk;
        p.pi[o] = pin;
        if (p.deriv) {
            // d/dz_k with the seed quantities fixed (d Delta_k / d z_k = 1)
            const double2 dpk = p.dpi[o], dpp = p.dpi_prev[o];
            const double2 dpin = cadd(cadd(cmul(alpha, pk), cmul(cadd(one, cmul(alpha, dl)), dpk)),
                                      cmul(c2, csub(dpk, dpp)));
            const double2 ip2 = cmul(ip, ip);
            const double2 num = cmul(csub(cmul(dpk, pin), cmul(pk, dpin)), ip2);
            sdak[k] = cmul(alpha, num);
            sdbk[k] = cmul(cmk(2.0 * beta.x, 2.0 * beta.y), cmul(ratio, num));
            sdip[k] = cmk(-cmul(dpin, ip2).x, -cmul(dpin, ip2).y);
            p.dpi_prev[o] = dpk;
            p.dpi[o] = dpin;
        }
        sak[k] = ak;
        sbk[k] = bk;
        sip[k] = ip;
        if (p.proj == PROJ_NONE) {
            p.ak[o] = ak;
            p.bk[o] = bk;
            p.ipi[o] = ip;
        }
        if (res <= p.tol) {
            p.conv_iter[o] = it + 1;
        } else {
            ++nunc;
            if (res > best) { best = res; bestk = k; }
        }
    }
    __syncthreads();
    if (p.proj != PROJ_NONE) {
        for (int e = tid; e < K * nfun; e += THREADS) {
            const int k = e / nfun, m = e % nfun;
            const double2 ip = sip[k];
            if (ip.x == 0.0 && ip.y == 0.0) continue;
            const size_t o = ((size_t)c * K + k) * p.M + m;
            const double2 u = p.u[o];
            if (p.deriv) {
                const double2 du = p.du[o];
                p.dt[o] = cadd(p.dt[o], cadd(cmul(sdak[k], u), cmul(sak[k], du)));
                p.du[o] = cadd(cadd(cmul(d[m], sdip[k]), cmul(sdbk[k], u)), cmul(sbk[k], du));
            }
            p.t[o] = cadd(p.t[o], cmul(sak[k], u));
            p.u[o] = cadd(cmul(d[m], ip), cmul(sbk[k], u));
        }
    }
    // block reductions: number of unconverged shifts, worst residual (ties -> lowest k)
    s_cnt[tid] = nunc;
    s_best[tid] = best;
    s_bestk[tid] = bestk;
    __syncthreads();
    for (int st = THREADS / 2; st >= 1; st >>= 1) {
        if (tid < st) {
            s_cnt[tid] += s_cnt[tid + st];
            const double ob = s_best[tid + st];
            const int ok = s_bestk[tid + st];
            if (ob > s_best[tid] || (ob == s_best[tid] && ok < s_bestk[tid])) {
                s_best[tid] = ob;
                s_bestk[tid] = ok;
            }
        }
        __syncthreads();
    }
    if (tid == 0) {
        ColState out = cs;
        out.iters = it + 1;
        out.n_unconv = s_cnt[0];
        if (out.n_unconv == 0) out.active = 0;
        int sw = 0;
        const int s2 = s_bestk[0];
        if (out.active && p.switching) {
            const bool seed_conv = p.conv_iter[(size_t)c * K + cs.seed] >= 0;
            const bool forced = p.force_switch_every > 0 && ((it + 1) % p.force_switch_every == 0);
            if ((seed_conv || forced) && s2 < K && s2 != cs.seed) sw = 1;
        }
        if (sw) {
            const double2 c1 = p.pi[(size_t)c * K + s2], c0 = p.pi_prev[(size_t)c * K + s2];
            out.rho = cdiv(cs.rho_new, cmul(c1, c1));
            out.alpha_prev = sak[s2];
            out.beta_prev = sbk[s2];
            out.sc_cur = cdiv(one, c1);
            out.sc_prev = cdiv(one, c0);
            out.zs = p.z[s2];
            out.seed = s2;
            out.switches += 1;
            s_c1 = c1;
            s_c0 = c0;
        } else {
            out.rho = cs.rho_new;
            out.alpha_prev = alpha;
            out.beta_prev = beta;
            out.sc_cur = one;
            out.sc_prev = one;
        }
        s_sw = sw;
        p.col[c] = out;
        if (out.active) atomicAdd(&p.flags[2], 1);
    }
    __syncthreads();
    if (s_sw) {
        const double2 c1 = s_c1, c0 = s_c0;
        for (int k = tid; k < K; k += THREADS) {
            const size_t o = (size_t)c * K + k;
            p.pi[o] = cdiv(p.pi[o], c1);
            p.pi_prev[o] = cdiv(p.pi_prev[o], c0);
            if (p.deriv) {
                p.dpi[o] = cdiv(p.dpi[o], c1);
                p.dpi_prev[o] = cdiv(p.dpi_prev[o], c0);
            }
        }
    }
}

// Full mode: x^k += alpha^k p^k, p^k = r'_{n+1}/pi^k_{n+1} + beta^k p^k.
__global__ void k_full_update(PanelDev p) {
    const int P = p.P;
    const long long per = (long long)p.npad * P;
    const long long items = per * p.K;
    for (long long idx = blockIdx.x * (long long)THREADS + threadIdx.x; idx < items;
         idx += (long long)gridDim.x * THREADS) {
        const int c = (int)(idx % P);
        const int k = (int)(idx / per);
        const size_t o = (size_t)c * p.K + k;
        const double2 ip = p.ipi[o];
        if (ip.x == 0.0 && ip.y == 0.0) continue;
        const double2 pk = p.Pk[idx];
        p.X[idx] = cadd(p.X[idx], cmul(p.ak[o], pk));
        p.Pk[idx] = cadd(cmul(p.Rp[idx % per], ip), cmul(p.bk[o], pk));
    }
}

__global__ void k_full_output(PanelDev p, const int32_t* __restrict__ orb2pad, int n_orb, int R, int ncols,
                              int c0, double2* __restrict__ out) {
    const long long items = (long long)p.K * ncols * n_orb;
    for (long long idx = blockIdx.x * (long long)THREADS + threadIdx.x; idx < items;
         idx += (long long)gridDim.x * THREADS) {
        const int o = (int)(idx % n_orb);
        const int c = (int)((idx / n_orb) % ncols);
        const int k = (int)(idx / ((long long)n_orb * ncols));
        out[((size_t)k * R + c0 + c) * n_orb + o] = p.X[((size_t)k * p.npad + orb2pad[o]) * p.P + c];
    }
}

// projected values src (p.t: G elements, p.dt: their z-derivatives) into the
// caller's layout out[(off[c] + m) * K + k]
__global__ void k_green_output(PanelDev p, int ncols, const int64_t* __restrict__ off, const double2* src,
                               double2* __restrict__ out) {
    const int c = blockIdx.x;
    if (c >= ncols) return;
    const int nf = p.col[c].nfun;
    for (int e = threadIdx.x; e < nf * p.K; e += THREADS) {
        const int m = e / p.K, k = e % p.K;
        out[(size_t)(off[c] + m) * p.K + k] = src[((size_t)c * p.K + k) * p.M + m];
    }
}

// Band energy and its gradients per projected element e = (a, b) of the
// H/S pattern (G_e(z_k) = G_ab, dG_e = dG_ab/dz):
//   e_terms[e] = -(g_s/pi) Im sum_k w_k z_k S_ab G_ab(z_k)   (E = sum_e e_terms)
//   gH[e] = -(g_s/pi) Im sum_k w_k z_k (-dG_ab)  = dE/dH_ba
//   gS[e] = -(g_s/pi) Im sum_k w_k (z_k G_ab + z_k^2 dG_ab) = dE/dS_ba
// (dG/dz = -G S G; G and G S G are symmetric, so (a, b) and (b, a) agree)
__global__ void k_band_energy_terms(const double2* __restrict__ G, const double2* __restrict__ dG,
                                    const double* __restrict__ S_el, int64_t n, int K, const double2* __restrict__ z,
                                    const double2* __restrict__ w, double g_s, double* __restrict__ e_terms,
                                    double* __restrict__ gH, double* __restrict__ gS) {
    const double f = -g_s / 3.14159265358979323846;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        double ae = 0.0, ah = 0.0, as = 0.0;
        for (int k = 0; k < K; ++k) {
            const double2 wz = cmul(w[k], z[k]);
            const double2 g = G[e * K + k], dg = dG[e * K + k];
            ae += cmul(wz, g).y;
            ah -= cmul(wz, dg).y;
            as += cmul(wz, g).y + cmul(cmul(wz, z[k]), dg).y;
        }
        e_terms[e] = f * S_el[e] * ae;
        gH[e] = f * ah;
        gS[e] = f * as;
    }
}

// Per projected element e = (a, b) of the pattern (G[e K + k] = G_ab(z_k)),
// the gradients of the charge-self-consistent free energy at fixed dq
// (Section 2.2, Eq. Hap-CSC; the contour grand potential Omega of the
// quadrature, whose H-derivative is the density matrix):
//   gH_e = rho_ab = -(g_s/pi) Im sum_k w_k G_ab(z_k)
//   gS_e = dOmega/dS_ab + rho_ab (V_I + V_J) / 2,
//   dOmega/dS_ab = (g_s/pi) Im sum_k w_k z_k G_ab(z_k),
// with V = gamma dq and I, J the atoms of orbitals a, b.
__global__ void k_csc_force_terms(const double2* __restrict__ G, int64_t n, int K, const double2* __restrict__ z,
                                  const double2* __restrict__ w, double g_s, const double* __restrict__ V,
                                  const int32_t* __restrict__ atom_a, const int32_t* __restrict__ atom_b,
                                  double* __restrict__ gH, double* __restrict__ gS) {
    const double f = g_s / 3.14159265358979323846;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        double ar = 0.0, az = 0.0;
        for (int k = 0; k < K; ++k) {
            const double2 g = G[e * K + k];
            ar += cmul(w[k], g).y;
            az += cmul(cmul(w[k], z[k]), g).y;
        }
        const double rho = -f * ar;
        gH[e] = rho;
        gS[e] = f * az + 0.5 * rho * (V[atom_a[e]] + V[atom_b[e]]);
    }
}

// Coulomb-gradient part of the charge-self-consistent forces:
// F_I -= dq_I sum_k (d gamma_Ik / d R_I) dq_k, dgamma [n][n][3]; one thread
// per atom, the k sum in index order.
__global__ void k_csc_force_coulomb(int n, const double* __restrict__ dgamma, const double* __restrict__ dq,
                                    double* __restrict__ F) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double g0 = 0.0, g1 = 0.0, g2 = 0.0;
        const double* row = dgamma + (size_t)i * n * 3;
        for (int k = 0; k < n; ++k) {
            g0 += row[3 * k] * dq[k];
            g1 += row[3 * k + 1] * dq[k];
            g2 += row[3 * k + 2] * dq[k];
        }
        F[3 * i] -= dq[i] * g0;
        F[3 * i + 1] -= dq[i] * g1;
        F[3 * i + 2] -= dq[i] * g2;
    }
}

// FMA throughput microbenchmark (measurement only): every thread runs
// `iters` rounds of 8 independent multiply-add chains on values that stay
// in registers (mode 0: scalar FP32 FMA, 1: packed FP32 FMA on float2, 2:
// FP64 FMA); the result is stored only if a run-time flag says so, which
// keeps the chains live without memory traffic.
__global__ void k_fma_peak(int mode, int iters, float a32, double a64, int store, float* out32, double* out64) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (mode == 2) {
        double v[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] = 1.0 + 1e-3 * (t + j);
        for (int i = 0; i < iters; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) v[j] = fma(v[j], a64, 1e-7);
        if (store) {
            double acc = 0.0;
#pragma unroll
            for (int j = 0; j < 8; ++j) acc += v[j];
            out64[t] = acc;
        }
    } else if (mode == 1) {
        float2 v[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] = make_float2(1.f + 1e-3f * j, 1.f - 1e-3f * j);
        const float2 a2 = make_float2(a32, a32), c2 = make_float2(1e-7f, 1e-7f);
        for (int i = 0; i < iters; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) v[j] = __ffma2_rn(v[j], a2, c2);
        if (store) {
            float acc = 0.f;
#pragma unroll
            for (int j = 0; j < 8; ++j) acc += v[j].x + v[j].y;
            out32[t] = acc;
        }
    } else {
        float v[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] = 1.f + 1e-3f * (t + j);
        for (int i = 0; i < iters; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) v[j] = fmaf(v[j], a32, 1e-7f);
        if (store) {
            float acc = 0.f;
#pragma unroll
            for (int j = 0; j < 8; ++j) acc += v[j];
            out32[t] = acc;
        }
    }
}

// out[0] = sum of v[0..n) in a fixed order (one CTA: strided partial sums,
// then a tree): deterministic whatever the launch history
__global__ void k_sum_fixed(const double* __restrict__ v, int64_t n, double* __restrict__ out) {
    __shared__ double red[THREADS];
    double acc = 0.0;
    for (long long i = threadIdx.x; i < n; i += THREADS) acc += v[i];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int st = THREADS / 2; st >= 1; st >>= 1) {
        if (threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = red[0];
}

// a7: q_j = -(g_s/pi) Im sum_k w_k s_j^T x_j(z_k)
__global__ void k_mulliken_output(PanelDev p, int ncols, const double2* __restrict__ w, double g_s,
                                  double* __restrict__ out) {
    __shared__ double red[THREADS];
    const int c = blockIdx.x;
    if (c >= ncols) return;
    double acc = 0.0;
    for (int k = threadIdx.x; k < p.K; k += THREADS) {
        const double2 tv = p.t[((size_t)c * p.K + k) * p.M];
        acc += w[k].x * tv.y + w[k].y * tv.x;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int st = THREADS / 2; st >= 1; st >>= 1) {
        if (threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[c] = -(g_s / 3.14159265358979323846) * red[0];
}

// ---------------------------------------------------------------------------
// Generalized Lanczos helpers (Section 3.2), one real vector stored in the
// real part of a P = 1 panel column.
// ---------------------------------------------------------------------------
// Generalized Lanczos on a panel of P columns (Section 3.2), one
// independent process per column; vectors [npad][P], real parts only.
// y = M x for M = H or S
__global__ void k_lz_spmv(DevSystem s, const double* __restrict__ M, const double2* __restrict__ x,
                          double2* __restrict__ y, int P) {
    const long long items = (long long)s.n_atoms * P;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < items;
         idx += (long long)gridDim.x * blockDim.x) {
        const int I = (int)(idx / P), c = (int)(idx % P);
        double acc[4] = {0.0, 0.0, 0.0, 0.0};
        for (int b = s.brow[I]; b < s.brow[I + 1]; ++b) {
            const int J = s.bcol[b];
            double xv[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) xv[e] = x[(size_t)(4 * J + e) * P + c].x;
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int e = 0; e < 4; ++e) acc[a] += M[16 * (size_t)b + 4 * a + e] * xv[e];
        }
#pragma unroll
        for (int a = 0; a < 4; ++a) y[(size_t)(4 * I + a) * P + c] = cmk(acc[a], 0.0);
    }
}

// out[c * stride] = x_c^T y_c (mode 0) or sqrt(x_c^T y_c) (mode 1)
__global__ void __launch_bounds__(THREADS) k_lz_dot(PanelDev p, const double2* __restrict__ x,
                                                    const double2* __restrict__ y, double* out, int stride, int mode) {
    __shared__ double smem[THREADS];
    const int P = p.P;
    double v[1] = {0.0};
    const long long items = (long long)p.npad * P;
    for (long long i = blockIdx.x * (long long)THREADS + threadIdx.x; i < items; i += (long long)gridDim.x * THREADS)
        v[0] += x[i].x * y[i].x;
    if (grid_reduce_cols<1>(v, P, p, smem)) {
        if (threadIdx.x < P) {
            const double t = smem[threadIdx.x];
            out[(size_t)threadIdx.x * stride] = (mode == 0) ? t : sqrt(fmax(t, 0.0));
        }
    }
}

// u_c = v_c / sqrt(n2_c), n2_c = v[row_c][c] = e_j^T S^-1 e_j (inactive columns: u = 0)
__global__ void k_lz_start(PanelDev p, const double2* __restrict__ v, double2* __restrict__ u, double* nrm2) {
    const int P = p.P;
    const long long items = (long long)p.npad * P;
    for (long long i = blockIdx.x * (long long)THREADS + threadIdx.x; i < items; i += (long long)gridDim.x * THREADS) {
        const int c = (int)(i % P);
        const ColState& cs = p.col[c];
        if (!cs.active) {
            u[i] = cmk(0.0, 0.0);
            continue;
        }
        const double n2 = v[(size_t)cs.row * P + c].x;
        u[i] = cmk(v[i].x / sqrt(n2), 0.0);
        if (i / P == 0) nrm2[c] = n2;
    }
}

// w = y - a_c u - b_c u_prev
__global__ void k_lz_combine(PanelDev p, const double2* __restrict__ y, const double2* __restrict__ u,
                             const double2* __restrict__ up, double2* __restrict__ w, const double* a,
                             const double* b, int sa, int sb) {
    const int P = p.P;
    const long long items = (long long)p.npad * P;
    for (long long i = blockIdx.x * (long long)THREADS + threadIdx.x; i < items; i += (long long)gridDim.x * THREADS) {
        const int c = (int)(i % P);
        w[i] = cmk(y[i].x - a[(size_t)c * sa] * u[i].x - b[(size_t)c * sb] * up[i].x, 0.0);
    }
}

// u_prev = u, u = w / b_c (0 when b_c = 0: invariant subspace found)
__global__ void k_lz_scale(PanelDev p, const double2* __restrict__ w, double2* __restrict__ u,
                           double2* __restrict__ up, const double* bnext, int sb) {
    const int P = p.P;
    const long long items = (long long)p.npad * P;
    for (long long i = blockIdx.x * (long long)THREADS + threadIdx.x; i < items; i += (long long)gridDim.x * THREADS) {
        const double bv = bnext[(size_t)(i % P) * sb];
        up[i] = u[i];
        u[i] = cmk(bv > 0.0 ? w[i].x / bv : 0.0, 0.0);
    }
}


// ---------------------------------------------------------------------------
// Charge self-consistency (Section 2.2, Eq. Hap-CSC)
// ---------------------------------------------------------------------------

// V_i = sum_k gamma_ik dq_k: one warp per row of gamma (coalesced), lanes
// add strided terms, then a fixed-order shuffle tree.
__global__ void k_csc_potential(const double* __restrict__ gamma, const double* __restrict__ dq, int n,
                                double* __restrict__ V) {
    const int lane = threadIdx.x & 31;
    const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long i = warp; i < n; i += nwarps) {
        const double* row = gamma + i * (long long)n;
        double acc = 0.0;
        for (int k = lane; k < n; k += 32) acc = fma(row[k], dq[k], acc);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) V[i] = acc;
    }
}

// H_IJ = H0_IJ + 1/2 S_IJ (V_I + V_J) for every stored block, with the FP32
// split (hi, lo) of the new H for the double-float products of the mixed
// path.  One warp per block row: the row's blocks are contiguous.  Padded
// orbital slots have S = 1 on the diagonal and no coupling; they only get
// V_I on their (decoupled) diagonal.
__global__ void k_csc_hamiltonian(DevSystem s, const double* __restrict__ H0, const double* __restrict__ V) {
    const int lane = threadIdx.x & 31;
    const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long I = warp; I < s.n_atoms; I += nwarps) {
        const double vI = V[I];
        const long long e0 = 16LL * s.brow[I], e1 = 16LL * s.brow[I + 1];
        for (long long e = e0 + lane; e < e1; e += 32) {
            const int J = s.bcol[e >> 4];
            const double h = H0[e] + 0.5 * s.S[e] * (vI + V[J]);
            s.H[e] = h;
            const float hi = (float)h;
            s.H32hi[e] = hi;
            s.H32lo[e] = (float)(h - (double)hi);
        }
    }
}

// q_atom[i] = sum of q_orb over the orbitals [orb_off[i], orb_off[i+1]) of atom i
__global__ void k_atom_sum(const double* __restrict__ q_orb, const int64_t* __restrict__ orb_off, int n_atoms,
                           double* __restrict__ q_atom) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n_atoms;
         i += (long long)gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int64_t o = orb_off[i]; o < orb_off[i + 1]; ++o) acc += q_orb[o];
        q_atom[i] = acc;
    }
}

// dq_out = q - q_ref, res = max_i |dq_out_i - dq_in_i| (as the bit pattern of
// a non-negative double: unsigned order is numeric order, and a NaN compares
// above +inf), dq_next = dq_in + mix (dq_out - dq_in).
__global__ void k_csc_mix(const double* __restrict__ q, const double* __restrict__ q_ref,
                          const double* __restrict__ dq_in, double* __restrict__ dq_next, double mix, int n,
                          unsigned long long* res_bits) {
    __shared__ unsigned long long smax[THREADS / 32];
    unsigned long long m = 0ull;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const double d = (q[i] - q_ref[i]) - dq_in[i];
        dq_next[i] = dq_in[i] + mix * d;
        const unsigned long long b = (unsigned long long)__double_as_longlong(fabs(d));
        m = b > m ? b : m;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long other = __shfl_xor_sync(0xffffffffu, m, o);
        m = other > m ? other : m;
    }
    if ((threadIdx.x & 31) == 0) smax[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = smax[w] > m ? smax[w] : m;
        atomicMax(res_bits, m);
    }
}


// G_r(z_k) = norm_r / (z_k - a_r0 - b_r1^2 / (z_k - a_r1 - ...)), one
// thread per (column r, point k), bottom-up (Section 3.2); a [R][n_steps],
// b [R][n_steps + 1], norm [R], G [R][K].
__global__ void k_lanczos_green(const double* __restrict__ a_all, const double* __restrict__ b_all,
                                const double* __restrict__ norm_all, int R, int n_steps, int K,
                                const double2* __restrict__ z, double2* __restrict__ G) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (long long)R * K;
         i += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(i / K), k = (int)(i % K);
        const double* a = a_all + (size_t)r * n_steps;
        const double* b = b_all + (size_t)r * (n_steps + 1);
        const double norm = norm_all[r];
        const double2 zk = z[k];
        double2 g = cmk(0.0, 0.0);
        for (int m = n_steps - 1; m >= 0; --m) {
            const double2 tail = (m + 1 < n_steps) ? cmk(b[m + 1] * b[m + 1] * g.x, b[m + 1] * b[m + 1] * g.y)
                                                   : cmk(0.0, 0.0);
            g = cdiv(cmk(1.0, 0.0), csub(cmk(zk.x - a[m], zk.y), tail));
        }
        G[i] = cmk(norm * g.x, norm * g.y);
    }
}


// ---------------------------------------------------------------------------
// Ragged batches: scatter one system's results into the caller's layout
// ---------------------------------------------------------------------------

// out[k][pos[c]][orb0 + o] = tmp[k][c][o]   (full solutions, [K][R][N])
__global__ void k_scatter_full(const double2* __restrict__ tmp, const int32_t* __restrict__ pos, int K, int Rq,
                               int64_t Nq, int R, int64_t N, int64_t orb0, double2* __restrict__ out) {
    const long long total = (long long)K * Rq * Nq;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long o = i % Nq;
        const long long kc = i / Nq;
        const int c = (int)(kc % Rq), k = (int)(kc / Rq);
        out[((long long)k * R + pos[c]) * N + orb0 + o] = tmp[i];
    }
}

// out[gidx[e] * K + k] = tmp[e * K + k]   (Green's function elements)
__global__ void k_scatter_rows(const double2* __restrict__ tmp, const int64_t* __restrict__ gidx, int64_t n, int K,
                               double2* __restrict__ out) {
    const long long total = n * (long long)K;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long e = i / K;
        out[gidx[e] * K + (i - e * K)] = tmp[i];
    }
}

// out[idx[e]] = v[e]
__global__ void k_scatter_values(const double* __restrict__ v, const int64_t* __restrict__ idx, int64_t n,
                                 double* __restrict__ out) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
        out[idx[e]] = v[e];
}

// out[pos[c]] = tmp[c]   (one value per column)
__global__ void k_scatter_cols(const double* __restrict__ tmp, const int32_t* __restrict__ pos, int Rq,
                               double* __restrict__ out) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < Rq; c += gridDim.x * blockDim.x) out[pos[c]] = tmp[c];
}


// ---------------------------------------------------------------------------
// Forces from the band-energy gradients (chain rule through the geometry)
// ---------------------------------------------------------------------------

// v_b = sum over the entries e of off-site block b = (I, J) of
// dE/dS_e dS_e/dd + dE/dH_e dH_e/dd (d = R_J - R_I); dH_dd == nullptr: the
// Eq. Hap-1 rule, dH_e/dd = K (eps_a + eps_b) / 2 dS_e/dd.  One warp per
// block row, lanes over its blocks.
__global__ void k_force_blocks(int n_atoms, const int* __restrict__ brow, const int* __restrict__ bcol,
                               const int64_t* __restrict__ boff, const int64_t* __restrict__ ooff,
                               const double* __restrict__ gH, const double* __restrict__ gS,
                               const double* __restrict__ dS_dd, const double* __restrict__ dH_dd,
                               const double* __restrict__ eps, double K, int64_t nvals, double* __restrict__ vblk) {
    const int lane = threadIdx.x & 31;
    const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long I = warp; I < n_atoms; I += nw) {
        const int ni = (int)(ooff[I + 1] - ooff[I]);
        for (int b = brow[I] + lane; b < brow[I + 1]; b += 32) {
            const int J = bcol[b];
            double v0 = 0.0, v1 = 0.0, v2 = 0.0;
            if (J != I) {
                const int nj = (int)(ooff[J + 1] - ooff[J]);
                for (int a = 0; a < ni; ++a)
                    for (int c = 0; c < nj; ++c) {
                        const int64_t e = boff[b] + (int64_t)a * nj + c;
                        double ws = gS[e], wh = gH[e];
                        if (dH_dd) {
                            v0 += ws * dS_dd[e] + wh * dH_dd[e];
                            v1 += ws * dS_dd[nvals + e] + wh * dH_dd[nvals + e];
                            v2 += ws * dS_dd[2 * nvals + e] + wh * dH_dd[2 * nvals + e];
                        } else {
                            const double w = ws + 0.5 * K * (eps[ooff[I] + a] + eps[ooff[J] + c]) * wh;
                            v0 += w * dS_dd[e];
                            v1 += w * dS_dd[nvals + e];
                            v2 += w * dS_dd[2 * nvals + e];
                        }
                    }
            }
            vblk[3 * (size_t)b] = v0;
            vblk[3 * (size_t)b + 1] = v1;
            vblk[3 * (size_t)b + 2] = v2;
        }
    }
}

// F_I = sum over off-site blocks (I, J) of v_(I,J) - v_(J,I), in block order
__global__ void k_force_atoms(int n_atoms, const int* __restrict__ brow, const int* __restrict__ bcol,
                              const int64_t* __restrict__ btrans, const double* __restrict__ vblk,
                              double* __restrict__ F) {
    for (long long I = blockIdx.x * (long long)blockDim.x + threadIdx.x; I < n_atoms;
         I += (long long)gridDim.x * blockDim.x) {
        double f0 = 0.0, f1 = 0.0, f2 = 0.0;
        for (int b = brow[I]; b < brow[I + 1]; ++b) {
            if (bcol[b] == I) continue;
            const int64_t t = btrans[b];
            f0 += vblk[3 * (size_t)b] - vblk[3 * (size_t)t];
            f1 += vblk[3 * (size_t)b + 1] - vblk[3 * (size_t)t + 1];
            f2 += vblk[3 * (size_t)b + 2] - vblk[3 * (size_t)t + 2];
        }
        F[3 * I] = f0;
        F[3 * I + 1] = f1;
        F[3 * I + 2] = f2;
    }
}


// r_0 = b for real right-hand sides b [ncols][n_orb] in caller orbital order
// (instead of e_j): written into Rcur and Rin at the padded slots
__global__ void k_panel_rhs(PanelDev p, const double* __restrict__ rhs, const int32_t* __restrict__ orb2pad,
                            int n_orb, int ncols) {
    const long long items = (long long)ncols * n_orb;
    for (long long i = blockIdx.x * (long long)THREADS + threadIdx.x; i < items; i += (long long)gridDim.x * THREADS) {
        const int c = (int)(i / n_orb), o = (int)(i % n_orb);
        const size_t e = (size_t)orb2pad[o] * p.P + c;
        const double2 v = cmk(rhs[i], 0.0);
        p.Rcur[e] = v;
        p.Rin[e] = v;
    }
}

// Mulliken vector-Jacobian product, one chunk of columns c0 .. c0+Rc-1 at a
// time: X[k][c][.] = G(z_k) e_c, Y[k][c][.] = G(z_k) s_c (caller order).
// For every stored entry (a, b):
//   Gamma_ba(z) = sum_c v_c Y[c]_b X[c]_a     ([G S D_v G]_ba, this chunk's share)
//   gH += -(g_s/pi) Im sum_k w_k Gamma_ba
//   gS += -(g_s/pi) Im sum_k w_k (v_b G_ba - z_k Gamma_ba), G_ba = X[a]_b when a is in the chunk
__global__ void k_vjp_accumulate(const double2* __restrict__ X, const double2* __restrict__ Y, int K, int Rc,
                                 int64_t N, const int32_t* __restrict__ cpos, const double* __restrict__ vc,
                                 const int32_t* __restrict__ ea, const int32_t* __restrict__ eb, int64_t ne,
                                 const double2* __restrict__ z,
                                 const double2* __restrict__ w, double g_s, double* __restrict__ gH,
                                 double* __restrict__ gS) {
    const double f = -g_s / 3.14159265358979323846;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < ne; e += (long long)gridDim.x * blockDim.x) {
        const int a = ea[e], b = eb[e];
        // position of column b in this chunk (-1: not one of its columns);
        // v_b G_ba = v_b (G e_b)_a, G being complex symmetric
        const int pb = cpos[b];
        double ah = 0.0, as = 0.0;
        for (int k = 0; k < K; ++k) {
            double2 gam = cmk(0.0, 0.0);
            for (int c = 0; c < Rc; ++c) {
                const size_t base = ((size_t)k * Rc + c) * N;
                gam = cadd(gam, cmul(cmk(vc[c], 0.0), cmul(Y[base + b], X[base + a])));
            }
            ah += cmul(w[k], gam).y;
            as -= cmul(cmul(w[k], z[k]), gam).y;
            if (pb >= 0) {
                const double2 gba = X[((size_t)k * Rc + pb) * N + a];
                as += vc[pb] * cmul(w[k], gba).y;
            }
        }
        gH[e] += f * ah;
        gS[e] += f * as;
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// launch accounting: a count of every kernel launch, and (when enabled) a
// pair of CUDA events around each launch on its own stream
// ---------------------------------------------------------------------------
namespace {
struct Profiler {
    // launch counts are atomics; the event pairs of the profiling mode and
    // the accumulated times are guarded by mu (host threads of one call
    // launch concurrently).  A pair is reused only after its stop event was
    // recorded and harvested; a thread's own harvest (after it synchronised
    // its stream) takes only the pairs it recorded, so it never waits for or
    // reads another thread's pairs in flight.
    std::mutex mu;
    bool on = false;
    std::vector<cudaEvent_t> ev;          // start/stop pairs
    std::vector<int> kid;                 // kernel id of each pair
    std::vector<std::thread::id> owner;   // thread that recorded the pair
    std::vector<size_t> free_pairs;
    std::vector<size_t> stopped;          // recorded, not yet harvested
    std::vector<char> in_graph;           // the pair is recorded by nodes of a captured graph
    std::atomic<int64_t> launches[K_COUNT] = {};
    double ms[K_COUNT] = {};
    std::atomic<int64_t> total{0};
    // launch intervals (ms after the reference event) per kernel class, for
    // the busy time when launches of several streams overlap
    cudaEvent_t ref = nullptr;
    bool ref_set = false;
    std::vector<std::pair<double, double>> iv[K_COUNT];
};
Profiler g_prof;

// set while this thread captures launches into a CUDA graph: they run (and
// are counted and timed) when the graph is launched
thread_local bool g_capturing = false;
// set while this thread captures an outer step (capture_step_*): every
// captured launch gets its own event pair, recorded by event nodes inside
// the graph, and is counted and timed at each launch of the graph
thread_local GraphProf* g_cap_prof = nullptr;
thread_local bool g_cap_timed = false;

static size_t new_pair_locked() {
    if (g_prof.free_pairs.empty()) {
        cudaEvent_t e[2];
        if (cudaEventCreate(&e[0]) != cudaSuccess || cudaEventCreate(&e[1]) != cudaSuccess) {
            cudaGetLastError();
            return (size_t)-1;
        }
        g_prof.ev.push_back(e[0]);
        g_prof.ev.push_back(e[1]);
        g_prof.kid.push_back(0);
        g_prof.owner.push_back(std::thread::id());
        g_prof.in_graph.push_back(0);
        g_prof.free_pairs.push_back(g_prof.kid.size() - 1);
    }
    const size_t pr = g_prof.free_pairs.back();
    g_prof.free_pairs.pop_back();
    return pr;
}

struct LaunchScope {
    cudaStream_t st;
    size_t pair = (size_t)-1;
    bool graph_pair = false;
    // count: kernels this launch runs (a graph launch runs several)
    LaunchScope(int id, cudaStream_t s, int count = 1) : st(s) {
        if (g_capturing) {
            if (!g_cap_prof) return;
            if (!g_cap_timed) {
                g_cap_prof->untimed_kid.push_back(id);
                g_cap_prof->untimed_counts.push_back(count);
                return;
            }
            std::lock_guard<std::mutex> lk(g_prof.mu);
            pair = new_pair_locked();
            if (pair == (size_t)-1) return;
            graph_pair = true;
            g_prof.kid[pair] = id;
            g_prof.in_graph[pair] = 1;
            g_cap_prof->pairs.push_back(pair);
            g_cap_prof->counts.push_back(count);
            // an external event node: the timestamp is taken at every replay
            cudaEventRecordWithFlags(g_prof.ev[2 * pair], st, cudaEventRecordExternal);
            return;
        }
        g_prof.total.fetch_add(count, std::memory_order_relaxed);
        g_prof.launches[id].fetch_add(count, std::memory_order_relaxed);
        if (!g_prof.on) return;
        std::lock_guard<std::mutex> lk(g_prof.mu);
        pair = new_pair_locked();
        if (pair == (size_t)-1) return;
        g_prof.kid[pair] = id;
        g_prof.owner[pair] = std::this_thread::get_id();
        cudaEventRecord(g_prof.ev[2 * pair], st);
    }
    ~LaunchScope() {
        if (pair == (size_t)-1) return;
        std::lock_guard<std::mutex> lk(g_prof.mu);
        if (graph_pair) {
            cudaEventRecordWithFlags(g_prof.ev[2 * pair + 1], st, cudaEventRecordExternal);
            return;
        }
        cudaEventRecord(g_prof.ev[2 * pair + 1], st);
        g_prof.stopped.push_back(pair);
    }
};

// all: every recorded pair (waits for them; call when no launch is in
// flight); else only the calling thread's pairs (complete after it
// synchronised its stream)
void harvest_locked(bool all) {
    std::vector<size_t> keep;
    const std::thread::id me = std::this_thread::get_id();
    for (size_t i : g_prof.stopped) {
        if (!all && g_prof.owner[i] != me) {
            keep.push_back(i);
            continue;
        }
        float t = 0.f, a = 0.f, b = 0.f;
        cudaEventSynchronize(g_prof.ev[2 * i + 1]);
        if (cudaEventElapsedTime(&t, g_prof.ev[2 * i], g_prof.ev[2 * i + 1]) == cudaSuccess)
            g_prof.ms[g_prof.kid[i]] += t;
        else
            cudaGetLastError();
        if (g_prof.ref_set && cudaEventElapsedTime(&a, g_prof.ref, g_prof.ev[2 * i]) == cudaSuccess &&
            cudaEventElapsedTime(&b, g_prof.ref, g_prof.ev[2 * i + 1]) == cudaSuccess)
            g_prof.iv[g_prof.kid[i]].push_back({(double)a, (double)b});
        else
            cudaGetLastError();
        if (!g_prof.in_graph[i]) g_prof.free_pairs.push_back(i);
    }
    g_prof.stopped.swap(keep);
}
}  // namespace

void profile_enable(bool on) {
    std::lock_guard<std::mutex> lk(g_prof.mu);
    harvest_locked(true);
    g_prof.on = on;
    for (int i = 0; i < K_COUNT; ++i) {
        g_prof.launches[i] = 0;
        g_prof.ms[i] = 0.0;
        g_prof.iv[i].clear();
    }
    g_prof.ref_set = false;
    if (on) {
        if (!g_prof.ref && cudaEventCreate(&g_prof.ref) != cudaSuccess) {
            cudaGetLastError();
            g_prof.ref = nullptr;
        }
        if (g_prof.ref && cudaEventRecord(g_prof.ref, 0) == cudaSuccess) g_prof.ref_set = true;
        else cudaGetLastError();
    }
}

void prof_harvest() {
    if (!g_prof.on) return;
    std::lock_guard<std::mutex> lk(g_prof.mu);
    harvest_locked(false);
}

void graph_prof_begin(GraphProf* gp) {
    g_capturing = true;
    // event pairs only while timing is on: otherwise the graph's launches are
    // counted (GraphProf::counts) but carry no event nodes
    g_cap_prof = gp;
    g_cap_timed = g_prof.on;
}
void graph_prof_end() {
    g_capturing = false;
    g_cap_prof = nullptr;
}

// At each launch of a graph captured with a GraphProf: its kernels are
// counted, and with profiling on its event pairs are queued for this
// thread's next harvest (after it synchronised the stream; a graph is
// launched again only after that).
void graph_prof_launched(const GraphProf& gp) {
    for (size_t i = 0; i < gp.pairs.size(); ++i) {
        g_prof.total.fetch_add(gp.counts[i], std::memory_order_relaxed);
        g_prof.launches[g_prof.kid[gp.pairs[i]]].fetch_add(gp.counts[i], std::memory_order_relaxed);
    }
    for (size_t i = 0; i < gp.untimed_kid.size(); ++i) {
        g_prof.total.fetch_add(gp.untimed_counts[i], std::memory_order_relaxed);
        g_prof.launches[gp.untimed_kid[i]].fetch_add(gp.untimed_counts[i], std::memory_order_relaxed);
    }
    if (!g_prof.on) return;
    std::lock_guard<std::mutex> lk(g_prof.mu);
    const std::thread::id me = std::this_thread::get_id();
    for (size_t pr : gp.pairs) {
        g_prof.owner[pr] = me;
        g_prof.stopped.push_back(pr);
    }
}

// The graph is gone: its pairs return to the pool (harvested first).
void graph_prof_release(GraphProf& gp) {
    std::lock_guard<std::mutex> lk(g_prof.mu);
    harvest_locked(true);
    for (size_t pr : gp.pairs) {
        g_prof.in_graph[pr] = 0;
        g_prof.free_pairs.push_back(pr);
    }
    gp.pairs.clear();
    gp.counts.clear();
    gp.untimed_kid.clear();
    gp.untimed_counts.clear();
}

void profile_read(int id, int64_t* launches, double* ms) {
    std::lock_guard<std::mutex> lk(g_prof.mu);
    harvest_locked(true);
    *launches = g_prof.launches[id];
    *ms = g_prof.ms[id];
}

int64_t launch_count() { return g_prof.total; }

double profile_busy(int id) {
    std::lock_guard<std::mutex> lk(g_prof.mu);
    harvest_locked(true);
    std::vector<std::pair<double, double>> v = g_prof.iv[id];
    std::sort(v.begin(), v.end());
    double busy = 0.0, lo = 0.0, hi = -1.0;
    for (const auto& x : v) {
        if (x.first > hi) {
            if (hi > lo) busy += hi - lo;
            lo = x.first;
            hi = x.second;
        } else if (x.second > hi) {
            hi = x.second;
        }
    }
    if (hi > lo) busy += hi - lo;
    return busy;
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
// TB_DF_RAG=0: systems with s-only atoms take the padded double-float SpMVs
static const bool g_df_rag = [] {
    const char* e = std::getenv("TB_DF_RAG");
    return !(e && std::atoi(e) == 0);
}();

static int gmax() {
    static const int g = [] {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        return 4 * (sms > 0 ? sms : 1);
    }();
    return g;
}

// Raise (never lower) a kernel's dynamic shared-memory limit: threads of a
// ragged batch may launch the same kernel with different sizes at once.
// The tracked limit starts at 0, so the attribute is always set explicitly:
// the 48 KB default covers static plus dynamic shared memory, and a size
// just under it can still be refused.
static bool ensure_dyn_smem(const void* kernel, size_t bytes, size_t& current) {
    static std::mutex mu;
    std::lock_guard<std::mutex> lk(mu);
    if (bytes <= current) return true;
    if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) != cudaSuccess)
        return false;
    current = bytes;
    return true;
}
int max_grid() { return gmax(); }

static int grid_for(long long items) {
    long long g = (items + THREADS - 1) / THREADS;
    int gm = gmax();
    return (int)(g < 1 ? 1 : (g > gm ? gm : g));
}

// Loads the kernels of the allocation-free Lanczos call onto the current
// device (cudaFuncGetAttributes loads a kernel that lazy module loading has
// not placed yet), so that the call's first launches need no device memory.
bool preload_noalloc_kernels() {
    const void* ks[] = {(const void*)k_panel_init, (const void*)k_inner_spmv, (const void*)k_inner_update,
                        (const void*)k_lz_start,   (const void*)k_lz_spmv,    (const void*)k_lz_dot,
                        (const void*)k_lz_combine, (const void*)k_lz_scale};
    for (const void* k : ks) {
        cudaFuncAttributes fa;
        if (cudaFuncGetAttributes(&fa, k) != cudaSuccess) return false;
    }
    return true;
}

void launch_split_f64(const double* v, float* hi, float* lo, long long n, cudaStream_t st) {
    LaunchScope ls_(K_OTHER, st);
    k_split_f64<<<grid_for(n), THREADS, 0, st>>>(v, hi, lo, n);
}
void launch_transpose_blocks(const float* in, float* out, long long nb, cudaStream_t st) {
    LaunchScope ls_(K_OTHER, st);
    k_transpose_blocks<<<grid_for(16 * nb), THREADS, 0, st>>>(in, out, nb);
}
void launch_compact_blocks(const DevSystem& s, cudaStream_t st) {
    LaunchScope ls_(K_OTHER, st);
    k_compact_blocks<<<grid_for(s.n_atoms), THREADS, 0, st>>>(s.n_atoms, s.brow, s.bcol, s.norb, s.S32, s.bmeta,
                                                               s.S32r);
}
void launch_ased_build(const DevSystem& s, const double* eps_pad, double K, cudaStream_t st) {
    {
        LaunchScope ls_(K_OTHER, st);
        k_ased_build<<<grid_for(s.n_atoms), THREADS, 0, st>>>(s.n_atoms, s.brow, s.bcol, s.S, s.H, eps_pad, K);
    }
}
void launch_panel_init(const DevSystem&, const PanelDev& p, cudaStream_t st) {
    {
        LaunchScope ls_(K_OTHER, st);
        k_panel_init<<<grid_for((long long)p.npad * p.P), THREADS, 0, st>>>(p);
    }
}
void launch_outer_spmm(const DevSystem& s, const PanelDev& p, bool sx_from_residual, cudaStream_t st) {
    {
        LaunchScope ls_(K_OUTER_SPMM, st);
        const bool rag = s.rag && g_df_rag;
        if (p.mixed && sx_from_residual && rag)
            k_outer_spmm<true, true, true><<<grid_for((long long)s.n_atoms * p.P), THREADS, 0, st>>>(s, p);
        else if (p.mixed && sx_from_residual)
            k_outer_spmm<true, true><<<grid_for((long long)s.n_atoms * p.P), THREADS, 0, st>>>(s, p);
        else if (p.mixed && rag)
            k_outer_spmm<true, false, true><<<grid_for((long long)s.n_atoms * p.P), THREADS, 0, st>>>(s, p);
        else if (p.mixed)
            k_outer_spmm<true><<<grid_for((long long)s.n_atoms * p.P), THREADS, 0, st>>>(s, p);
        else
            k_outer_spmm<false><<<grid_for((long long)s.n_atoms * p.P), THREADS, 0, st>>>(s, p);
    }
}
void launch_outer_update(const DevSystem&, const PanelDev& p, cudaStream_t st) {
    {
        LaunchScope ls_(K_OUTER_UPDATE, st);
        k_outer_update<<<grid_for((long long)p.npad * p.P), THREADS, 0, st>>>(p);
    }
}
void launch_inner_spmv(const DevSystem& s, const PanelDev& p, int it, cudaStream_t st) {
    {
        LaunchScope ls_(K_INNER_SPMV, st);
        k_inner_spmv<<<grid_for((long long)s.n_atoms * p.P), THREADS, 0, st>>>(s, p, it);
    }
}
void launch_inner_update(const DevSystem&, const PanelDev& p, int it, cudaStream_t st) {
    {
        LaunchScope ls_(K_INNER_UPDATE, st);
        k_inner_update<<<grid_for((long long)p.npad * p.P), THREADS, 0, st>>>(p, it);
    }
}
void launch_finish(const DevSystem&, const PanelDev& p, cudaStream_t st) {
    {
        LaunchScope ls_(K_FINISH, st);
        k_finish<<<grid_for((long long)p.npad * p.P), THREADS, 0, st>>>(p);
    }
}
void launch_refine_start(const DevSystem&, const PanelDev& p, const double2* b, cudaStream_t st) {
    LaunchScope ls_(K_REFINE_AUX, st);
    k_refine_start<<<grid_for((long long)p.npad * p.P), THREADS, 0, st>>>(p, b);
}
void launch_refine_residual(const DevSystem& s, const PanelDev& p, const double2* b, cudaStream_t st, bool fp64) {
    LaunchScope ls_(K_REFINE_RESIDUAL, st);
    if (fp64)   // FP64 products; columns already within inner_tol exit at once
        k_refine_residual<false><<<grid_for((long long)s.n_atoms * p.P), THREADS, 0, st>>>(s, p, b);
    else if (s.rag && g_df_rag)
        k_refine_residual<true, true><<<grid_for((long long)s.n_atoms * p.P), THREADS, 0, st>>>(s, p, b);
    else
        k_refine_residual<true><<<grid_for((long long)s.n_atoms * p.P), THREADS, 0, st>>>(s, p, b);
}
void launch_refine_scale(const DevSystem&, const PanelDev& p, const double2* src, float cheb_gamma, cudaStream_t st) {
    LaunchScope ls_(K_REFINE_AUX, st);
    k_refine_scale<<<grid_for((long long)p.npad * p.P), THREADS, 0, st>>>(p, src, cheb_gamma);
}
void launch_split_panel(const PanelDev& p, cudaStream_t st) {
    LaunchScope ls_(K_REFINE_AUX, st);
    k_split_panel<<<grid_for((long long)p.npad * p.P), THREADS, 0, st>>>(p);
}
void launch_refine_add(const DevSystem&, const PanelDev& p, cudaStream_t st) {
    LaunchScope ls_(K_REFINE_AUX, st);
    k_refine_add<<<grid_for((long long)p.npad * p.P), THREADS, 0, st>>>(p);
}
size_t inner32_grp_smem(const DevSystem& s) {
    const size_t xregion = (size_t)s.max_union * 4 * PC * sizeof(float2);
    const size_t red_bytes = (size_t)(s.grpG * PC / 2 / 32) * (PC / 2) * 8 * sizeof(double);
    return GRP_HDR + (xregion > red_bytes ? xregion : red_bytes) + (size_t)s.max_gblocks * 64;
}

void launch_inner32_spmv(const DevSystem& s, const PanelDev& p, int it, cudaStream_t st) {
    LaunchScope ls_(K_INNER32_SPMV, st);
    // the grouped form wins on narrow panels (measured on the Si 4096-atom
    // system: 28 vs 35 us at 64 columns); from 128 columns on, the
    // register-gather form with its higher occupancy is faster
    if (s.grpG > 0 && p.P >= PC && p.P <= 64) {
        const size_t sm = inner32_grp_smem(s);
        static const bool attr = [] {
            // the dynamic limit leaves room for the kernel's static shared memory
            cudaFuncAttributes fa;
            return cudaFuncGetAttributes(&fa, k_inner32_spmv_grp) == cudaSuccess &&
                   cudaFuncSetAttribute(k_inner32_spmv_grp, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        227 * 1024 - (int)fa.sharedSizeBytes) == cudaSuccess &&
                   cudaFuncSetAttribute(k_inner32_spmv_grp, cudaFuncAttributePreferredSharedMemoryCarveout, 100) ==
                       cudaSuccess;
        }();
        (void)attr;
        k_inner32_spmv_grp<<<s.n_groups * (p.P / PC), s.grpG * (PC / 2), sm, st>>>(s, p, it);
    } else if (p.P >= 2) {
        const int g = grid_for((long long)s.n_atoms * (p.P / 2));
        switch (p.P) {
            case 256: k_inner32_spmv<2, 256><<<g, THREADS, 0, st>>>(s, p, it); break;
            case 128: k_inner32_spmv<2, 128><<<g, THREADS, 0, st>>>(s, p, it); break;
            case 64: k_inner32_spmv<2, 64><<<g, THREADS, 0, st>>>(s, p, it); break;
            case 32: k_inner32_spmv<2, 32><<<g, THREADS, 0, st>>>(s, p, it); break;
            case 16: k_inner32_spmv<2, 16><<<g, THREADS, 0, st>>>(s, p, it); break;
            case 8: k_inner32_spmv<2, 8><<<g, THREADS, 0, st>>>(s, p, it); break;
            case 4: k_inner32_spmv<2, 4><<<g, THREADS, 0, st>>>(s, p, it); break;
            default: k_inner32_spmv<2><<<g, THREADS, 0, st>>>(s, p, it); break;
        }
    }
    else
        k_inner32_spmv<1><<<grid_for((long long)s.n_atoms * p.P), THREADS, 0, st>>>(s, p, it);
}
// TB_CHEB_CPT=2 / 4 forces the two- or four-columns-per-thread form of the
// Chebyshev step (panels narrower than 4 columns always take the two-column
// form); tb_autotune's choice for the call's size class comes first
static const int g_cheb_cpt_env = [] {
    const char* e = std::getenv("TB_CHEB_CPT");
    return e ? std::atoi(e) : 0;
}();

// TB_CHEB_RAG=0: systems with s-only atoms also take the padded form
static const bool g_cheb_rag = [] {
    const char* e = std::getenv("TB_CHEB_RAG");
    return !(e && std::atoi(e) == 0);
}();

template <bool LAST>
static void cheb4_launch(const DevSystem& s, const PanelDev& p, const float2* cur, float2* io, float omega,
                         float gamma, int mode, cudaStream_t st) {
    const int g = std::min(grid_for((long long)s.n_atoms * (p.P / 4)), 3 * (gmax() / 4));
    if (s.rag && g_cheb_rag) {
        switch (p.P) {
            case 256: k_inner32_cheb4r<256, LAST><<<g, THREADS, 0, st>>>(s, p, cur, io, omega, gamma, mode); break;
            case 128: k_inner32_cheb4r<128, LAST><<<g, THREADS, 0, st>>>(s, p, cur, io, omega, gamma, mode); break;
            case 64: k_inner32_cheb4r<64, LAST><<<g, THREADS, 0, st>>>(s, p, cur, io, omega, gamma, mode); break;
            default: k_inner32_cheb4r<0, LAST><<<g, THREADS, 0, st>>>(s, p, cur, io, omega, gamma, mode); break;
        }
        return;
    }
    switch (p.P) {
        case 256: k_inner32_cheb4<256, LAST><<<g, THREADS, 0, st>>>(s, p, cur, io, omega, gamma, mode); break;
        case 128: k_inner32_cheb4<128, LAST><<<g, THREADS, 0, st>>>(s, p, cur, io, omega, gamma, mode); break;
        case 64: k_inner32_cheb4<64, LAST><<<g, THREADS, 0, st>>>(s, p, cur, io, omega, gamma, mode); break;
        default: k_inner32_cheb4<0, LAST><<<g, THREADS, 0, st>>>(s, p, cur, io, omega, gamma, mode); break;
    }
}

template <bool LAST>
static void cheb_launch(const DevSystem& s, const PanelDev& p, const float2* cur, float2* io, float omega,
                        float gamma, int mode, cudaStream_t st) {
    // default form: four columns per thread (measured best on the silicon
    // benchmark and on ragged water batches, whose concurrent systems fill
    // the GPU; a small system solved alone runs faster with two, which
    // tb_autotune finds for its size class), two for narrow panels
    // (measured on the 100 000-atom crystal: at 4 and 8 columns per panel the
    // two-column form's twice as many threads win, 61 / 69 against 93 /
    // 100 us per step; from 16 columns on, four columns per thread)
    const int cpt = p.cheb_cpt ? p.cheb_cpt : g_cheb_cpt_env ? g_cheb_cpt_env : (p.P >= 16 ? 4 : 2);
    if (cpt == 4 && p.P >= 4) {
        cheb4_launch<LAST>(s, p, cur, io, omega, gamma, mode, st);
        return;
    }

    if (p.P >= 2) {
        const int g = grid_for((long long)s.n_atoms * (p.P / 2));
        switch (p.P) {
            case 256: k_inner32_cheb<2, 256, LAST><<<g, THREADS, 0, st>>>(s, p, cur, io, omega, gamma, mode); break;
            case 128: k_inner32_cheb<2, 128, LAST><<<g, THREADS, 0, st>>>(s, p, cur, io, omega, gamma, mode); break;
            case 64: k_inner32_cheb<2, 64, LAST><<<g, THREADS, 0, st>>>(s, p, cur, io, omega, gamma, mode); break;
            case 32: k_inner32_cheb<2, 32, LAST><<<g, THREADS, 0, st>>>(s, p, cur, io, omega, gamma, mode); break;
            case 16: k_inner32_cheb<2, 16, LAST><<<g, THREADS, 0, st>>>(s, p, cur, io, omega, gamma, mode); break;
            case 8: k_inner32_cheb<2, 8, LAST><<<g, THREADS, 0, st>>>(s, p, cur, io, omega, gamma, mode); break;
            case 4: k_inner32_cheb<2, 4, LAST><<<g, THREADS, 0, st>>>(s, p, cur, io, omega, gamma, mode); break;
            default: k_inner32_cheb<2, 0, LAST><<<g, THREADS, 0, st>>>(s, p, cur, io, omega, gamma, mode); break;
        }
    } else {
        k_inner32_cheb<1, 0, LAST><<<grid_for((long long)s.n_atoms * p.P), THREADS, 0, st>>>(s, p, cur, io, omega,
                                                                                          gamma, mode);
    }
}
void launch_inner32_cheb(const DevSystem& s, const PanelDev& p, const float2* cur, float2* io, float omega,
                         float gamma, int mode, cudaStream_t st) {
    LaunchScope ls_(K_INNER32_CHEB, st);
    if (mode == 2) cheb_launch<true>(s, p, cur, io, omega, gamma, mode, st);
    else cheb_launch<false>(s, p, cur, io, omega, gamma, mode, st);
}

// Steps 1 .. n-1 of a Chebyshev round as one CUDA graph: the launches of a
// round have the same arguments in every round of a panel (the kernels read
// the round's state from device memory), so they are captured once, on a
// private stream (the caller's may be the legacy default stream, which
// cannot be captured), and replayed with one launch per round.
bool cheb_graph_build(const DevSystem& s, const PanelDev& p, const float* omega, int n, float gamma,
                      cudaGraphExec_t* out) {
    *out = nullptr;
    cudaStream_t cs;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    cudaGraph_t g = nullptr;
    bool ok = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
        g_capturing = true;
        for (int k = 1; k < n; ++k) {
            const float2* cur = (k & 1) ? p.x32 : p.p32;
            float2* io = (k & 1) ? p.p32 : p.x32;
            const int mode = k == n - 1 ? 2 : (k == 1 ? 1 : 0);
            launch_inner32_cheb(s, p, cur, io, omega[k], gamma, mode, cs);
        }
        g_capturing = false;
        ok = cudaStreamEndCapture(cs, &g) == cudaSuccess && g != nullptr;
    }
    if (ok) ok = cudaGraphInstantiate(out, g, 0) == cudaSuccess;
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    if (!ok) {
        cudaGetLastError();
        *out = nullptr;
    }
    return ok;
}
void cheb_graph_launch(cudaGraphExec_t g, int steps, cudaStream_t st) {
    LaunchScope ls_(K_INNER32_CHEB, st, steps);
    cudaGraphLaunch(g, st);
}
void cheb_graph_destroy(cudaGraphExec_t g) {
    if (g) cudaGraphExecDestroy(g);
}
void launch_inner32_update(const DevSystem&, const PanelDev& p, int it, cudaStream_t st) {
    LaunchScope ls_(K_INNER32_UPDATE, st);
    if (p.P >= 2)
        k_inner32_update<2><<<grid_for((long long)p.npad * p.P / 2), THREADS, 0, st>>>(p, it);
    else
        k_inner32_update<1><<<grid_for((long long)p.npad * p.P), THREADS, 0, st>>>(p, it);
}
static size_t shift_smem(const PanelDev& p) {
    return sizeof(double2) * ((size_t)(p.M > 0 ? p.M : 1) + (p.deriv ? 6 : 3) * (size_t)p.K);
}
void launch_shift_init(const DevSystem& s, const PanelDev& p, cudaStream_t st) {
    const size_t sm = shift_smem(p);
    static size_t lim_init = 0;
    ensure_dyn_smem((const void*)k_shift_init, sm, lim_init);
    {
        LaunchScope ls_(K_OTHER, st);
        k_shift_init<<<p.P, THREADS, sm, st>>>(s, p);
    }
    if (p.proj == PROJ_NONE) {
        LaunchScope ls_(K_OTHER, st);
        k_full_init<<<grid_for((long long)p.npad * p.P * p.K), THREADS, 0, st>>>(p);
    }
}
void launch_shift_step(const DevSystem& s, const PanelDev& p, cudaStream_t st) {
    const size_t sm = shift_smem(p);
    static size_t lim_step = 0;
    ensure_dyn_smem((const void*)k_shift_step, sm, lim_step);
    {
        LaunchScope ls_(K_SHIFT_STEP, st);
        k_shift_step<<<p.P, THREADS, sm, st>>>(s, p);
    }
}
void launch_full_update(const DevSystem&, const PanelDev& p, cudaStream_t st) {
    {
        LaunchScope ls_(K_FULL_UPDATE, st);
        k_full_update<<<grid_for((long long)p.npad * p.P * p.K), THREADS, 0, st>>>(p);
    }
}
void launch_full_output(const PanelDev& p, const int32_t* orb2pad, int n_orb, int R, int ncols, int c0,
                        double2* out, cudaStream_t st) {
    {
        LaunchScope ls_(K_OTHER, st);
        k_full_output<<<grid_for((long long)p.K * ncols * n_orb), THREADS, 0, st>>>(p, orb2pad, n_orb, R, ncols, c0, out);
    }
}
void launch_green_output(const PanelDev& p, int ncols, const int64_t* off, double2* out, cudaStream_t st) {
    {
        LaunchScope ls_(K_OTHER, st);
        k_green_output<<<p.P, THREADS, 0, st>>>(p, ncols, off, p.t, out);
    }
}
void launch_green_deriv_output(const PanelDev& p, int ncols, const int64_t* off, double2* out, cudaStream_t st) {
    LaunchScope ls_(K_OTHER, st);
    k_green_output<<<p.P, THREADS, 0, st>>>(p, ncols, off, p.dt, out);
}
void launch_band_energy_terms(const double2* G, const double2* dG, const double* S_el, int64_t n, int K,
                              const double2* z, const double2* w, double g_s, double* e_terms, double* gH,
                              double* gS, cudaStream_t st) {
    LaunchScope ls_(K_OTHER, st);
    k_band_energy_terms<<<grid_for(n), THREADS, 0, st>>>(G, dG, S_el, n, K, z, w, g_s, e_terms, gH, gS);
}
void launch_csc_force_terms(const double2* G, int64_t n, int K, const double2* z, const double2* w, double g_s,
                            const double* V, const int32_t* atom_a, const int32_t* atom_b, double* gH, double* gS,
                            cudaStream_t st) {
    LaunchScope ls_(K_CSC, st);
    k_csc_force_terms<<<grid_for(n), THREADS, 0, st>>>(G, n, K, z, w, g_s, V, atom_a, atom_b, gH, gS);
}
void launch_csc_force_coulomb(int n, const double* dgamma, const double* dq, double* F, cudaStream_t st) {
    LaunchScope ls_(K_CSC, st);
    k_csc_force_coulomb<<<grid_for(n), THREADS, 0, st>>>(n, dgamma, dq, F);
}
void launch_fma_peak(int mode, int blocks, int threads, int iters, float* out32, double* out64, cudaStream_t st) {
    LaunchScope ls_(K_OTHER, st);
    k_fma_peak<<<blocks, threads, 0, st>>>(mode, iters, 0.999999f, 0.999999999, 0, out32, out64);
}
void launch_sum_fixed(const double* v, int64_t n, double* out, cudaStream_t st) {
    LaunchScope ls_(K_OTHER, st);
    k_sum_fixed<<<1, THREADS, 0, st>>>(v, n, out);
}
void launch_mulliken_output(const PanelDev& p, int ncols, const double2* w, double g_s, double* out,
                            cudaStream_t st) {
    {
        LaunchScope ls_(K_OTHER, st);
        k_mulliken_output<<<p.P, THREADS, 0, st>>>(p, ncols, w, g_s, out);
    }
}
void launch_lz_spmv(const DevSystem& s, const double* M, const double2* x, double2* y, int P, cudaStream_t st) {
    LaunchScope ls_(K_OTHER, st);
    k_lz_spmv<<<grid_for((long long)s.n_atoms * P), THREADS, 0, st>>>(s, M, x, y, P);
}
void launch_lz_dot(const PanelDev& p, const double2* x, const double2* y, double* out, int stride, int mode,
                   cudaStream_t st) {
    LaunchScope ls_(K_OTHER, st);
    k_lz_dot<<<grid_for((long long)p.npad * p.P), THREADS, 0, st>>>(p, x, y, out, stride, mode);
}
void launch_lz_combine(const PanelDev& p, const double2* y, double2* u, double2* u_prev, double2* w,
                       const double* a, const double* b, int sa, int sb, cudaStream_t st) {
    LaunchScope ls_(K_OTHER, st);
    k_lz_combine<<<grid_for((long long)p.npad * p.P), THREADS, 0, st>>>(p, y, u, u_prev, w, a, b, sa, sb);
}
void launch_lz_scale(const PanelDev& p, double2* w, double2* u, double2* u_prev, const double* bnext, int sb,
                     cudaStream_t st) {
    LaunchScope ls_(K_OTHER, st);
    k_lz_scale<<<grid_for((long long)p.npad * p.P), THREADS, 0, st>>>(p, w, u, u_prev, bnext, sb);
}
void launch_lz_start(const PanelDev& p, const double2* v, double2* u, double* nrm2, cudaStream_t st) {
    LaunchScope ls_(K_OTHER, st);
    k_lz_start<<<grid_for((long long)p.npad * p.P), THREADS, 0, st>>>(p, v, u, nrm2);
}


void launch_csc_potential(const double* gamma, const double* dq, int n, double* V, cudaStream_t st) {
    LaunchScope ls_(K_CSC, st);
    k_csc_potential<<<grid_for((long long)n * 32), THREADS, 0, st>>>(gamma, dq, n, V);
}

void launch_csc_hamiltonian(const DevSystem& s, const double* H0, const double* V, cudaStream_t st) {
    LaunchScope ls_(K_CSC, st);
    k_csc_hamiltonian<<<grid_for((long long)s.n_atoms * 32), THREADS, 0, st>>>(s, H0, V);
}

void launch_atom_sum(const double* q_orb, const int64_t* orb_off, int n_atoms, double* q_atom, cudaStream_t st) {
    LaunchScope ls_(K_CSC, st);
    k_atom_sum<<<grid_for(n_atoms), THREADS, 0, st>>>(q_orb, orb_off, n_atoms, q_atom);
}

void launch_csc_mix(const double* q, const double* q_ref, const double* dq_in, double* dq_next, double mix, int n,
                    unsigned long long* res_bits, cudaStream_t st) {
    LaunchScope ls_(K_CSC, st);
    k_csc_mix<<<grid_for(n), THREADS, 0, st>>>(q, q_ref, dq_in, dq_next, mix, n, res_bits);
}


void launch_lanczos_green(const double* a, const double* b, const double* norm, int R, int n_steps, int K,
                          const double2* z, double2* G, cudaStream_t st) {
    LaunchScope ls_(K_OTHER, st);
    k_lanczos_green<<<grid_for((long long)R * K), THREADS, 0, st>>>(a, b, norm, R, n_steps, K, z, G);
}


void launch_scatter_full(const double2* tmp, const int32_t* pos, int K, int Rq, int64_t Nq, int R, int64_t N,
                         int64_t orb0, double2* out, cudaStream_t st) {
    LaunchScope ls_(K_OTHER, st);
    k_scatter_full<<<grid_for((long long)K * Rq * Nq), THREADS, 0, st>>>(tmp, pos, K, Rq, Nq, R, N, orb0, out);
}

void launch_scatter_rows(const double2* tmp, const int64_t* gidx, int64_t n, int K, double2* out, cudaStream_t st) {
    LaunchScope ls_(K_OTHER, st);
    k_scatter_rows<<<grid_for(n * (long long)K), THREADS, 0, st>>>(tmp, gidx, n, K, out);
}

void launch_scatter_values(const double* v, const int64_t* idx, int64_t n, double* out, cudaStream_t st) {
    LaunchScope ls_(K_OTHER, st);
    k_scatter_values<<<grid_for(n), THREADS, 0, st>>>(v, idx, n, out);
}

void launch_scatter_cols(const double* tmp, const int32_t* pos, int Rq, double* out, cudaStream_t st) {
    LaunchScope ls_(K_OTHER, st);
    k_scatter_cols<<<grid_for(Rq), THREADS, 0, st>>>(tmp, pos, Rq, out);
}


void launch_force_blocks(int n_atoms, const int* brow, const int* bcol, const int64_t* boff, const int64_t* ooff,
                         const double* gH, const double* gS, const double* dS_dd, const double* dH_dd,
                         const double* eps, double K, int64_t nvals, double* vblk, cudaStream_t st) {
    LaunchScope ls_(K_OTHER, st);
    k_force_blocks<<<grid_for((long long)n_atoms * 32), THREADS, 0, st>>>(n_atoms, brow, bcol, boff, ooff, gH, gS,
                                                                           dS_dd, dH_dd, eps, K, nvals, vblk);
}

void launch_force_atoms(int n_atoms, const int* brow, const int* bcol, const int64_t* btrans, const double* vblk,
                        double* F, cudaStream_t st) {
    LaunchScope ls_(K_OTHER, st);
    k_force_atoms<<<grid_for(n_atoms), THREADS, 0, st>>>(n_atoms, brow, bcol, btrans, vblk, F);
}


void launch_panel_rhs(const PanelDev& p, const double* rhs, const int32_t* orb2pad, int n_orb, int ncols,
                      cudaStream_t st) {
    LaunchScope ls_(K_OTHER, st);
    k_panel_rhs<<<grid_for((long long)ncols * n_orb), THREADS, 0, st>>>(p, rhs, orb2pad, n_orb, ncols);
}

void launch_vjp_accumulate(const double2* X, const double2* Y, int K, int Rc, int64_t N, const int32_t* cpos,
                           const double* vc, const int32_t* ea, const int32_t* eb, int64_t ne,
                           const double2* z, const double2* w, double g_s, double* gH, double* gS, cudaStream_t st) {
    LaunchScope ls_(K_OTHER, st);
    k_vjp_accumulate<<<grid_for(ne), THREADS, 0, st>>>(X, Y, K, Rc, N, cpos, vc, ea, eb, ne, z, w, g_s, gH, gS);
}

}  // namespace tb
