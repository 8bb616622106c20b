// Shared-basis Lanczos kernel for sm_103a: all K shifted solves of a rational
// evaluation (Eq. (5) of Rittich & Speck, arXiv:1912.03312) on one Krylov
// basis of B = tau (H - c), one grid barrier per Krylov step.
//
// Krylov step j (one sweep; every tile CTA, own tile plus a one-point halo):
//
//   u_j  = s_j (w'_{j-1} - alpha_{j-1} u_{j-1} - beta_{j-1} u_{j-2})   (pointwise,
//          recomputed on the halo from the stored vectors so no second barrier
//          is needed before the stencil; w' = B u / f, f = |first stencil
//          coefficient|)
//   w'_j = B u_j / f                          (stencil from shared memory)
//   partial sums of ||u_j||^2 and Re u_j^H w'_j
//
// The inputs of the update (w'_{j-1}, u_{j-1}, u_{j-2} on the tile and its
// halo, the diagonal on the tile) are staged in shared memory by asynchronous
// copies issued as soon as the barrier opens, while the CTA reduces the
// partials; the inner products are compensated sums of FP32 hi/lo pieces
// (about 1e-13 relative; the FP64 pipe stays free for the recurrence; sweep 0,
// on the caller's state of any scale, sums in FP64).  In the double-float mode
// (LzArgs::df) the recurrence itself, from u_1 on, runs in pairs of floats on
// the FP32 pipe as well (the section on that mode below).  Every CTA reduces the
// partials in FP64 in the same fixed order and derives the same coefficients:
// with n_j = ||u_j||^2, alpha_j = Re u_j^H w'_j / n_j (f alpha_j is the
// Rayleigh quotient of B, real because B is real symmetric) and beta_j = n_j /
// (s_j n_{j-1}), which makes the tridiagonal matrix symmetric.  With q_j = u_j
// / ||u_j|| the recurrence reads
//
//   B q_j = T(j+1, j) q_{j+1} + T(j, j) q_j + T(j, j-1) q_{j-1},
//   T(j, j) = f alpha_j,  T(j+1, j) = f sqrt(n_{j+1} / n_j) / s_{j+1},
//
// exactly for the coefficients used (whatever the accuracy of the inner
// products that chose them), so B Q_k = Q_{k+1} T_k holds to the rounding of
// the recurrence (FP64, or double-float pairs on the FP32 pipe in the
// double-float mode) with T_k tridiagonal.  The scale s_j is one (two fused
// multiply-adds per component) while n stays within [2^-30, 2^30], else the
// power of two that brings u_j back to unit scale.  The shifted systems (B - s_k I) x = psi share
// Q_k (Sec. 5 of the paper: the Krylov spaces of shifted systems coincide);
// pole k minimises ||beta e_1 - (T_k - s_k [I; 0]) y|| by its own Givens
// rotations (GMRES on the shared basis).  The columns are unit vectors but
// orthogonal only locally, so the stop uses the bound ||r_k|| = ||Q_{k+1} z||
// <= ||z||_1 = |g_{k+1}| L_k, z the residual's coordinates (the rotations
// applied backwards to g_{k+1} e_{k+1}), L_k = c_k + |s_k| L_{k-1} <= sqrt(k+1)
// (times a 1e-4 margin for the computed norms).
//
// CTA 0 is the control CTA: it owns no tiles, runs the per-pole Givens
// recurrences one step behind the sweeps, and once every pole has met its
// bound stops the iteration and back-substitutes y_k in the same step (while
// the tile CTAs run the sweep whose result is not needed).  The result of the
// evaluation is psi' = alpha_0 psi + sum_k alpha_k Q y_k = alpha_0 psi +
// Q (sum_k alpha_k y_k): one pass over the basis (the pole sum of Eq. (5)).
#include <cuda_runtime.h>

#include <algorithm>

#include "devsync.cuh"
#include "lanczos.h"

namespace rexi {

namespace {

using dev::global_ns;
using dev::grid_sync;

// This CTA's index within its problem's range of CTAs, and the range's size.
__device__ __forceinline__ int lz_bid(const LzArgs& A) { return (int)blockIdx.x - A.cta0; }
__device__ __forceinline__ int lz_nct(const LzArgs& A) { return A.ncta; }

constexpr int kLzWarps = kLzBlock / 32;
constexpr int kErrInternal = -3;        // REXI_ECUDA: the iteration outran its workspace

// ---- index checks (builds with REXI_DEBUG defined) --------------------------
//
// LZ_OK(i, extent, site) is true when 0 <= i < extent; LZ_AT(base, i, extent,
// site) is base[i] then.  A failed check records the first failure (site,
// index, extent) and a count in A.dbg, sets the launch's error word to
// REXI_EBOUNDS and skips the access (LZ_AT redirects it to a scratch slot), so
// nothing outside a buffer is touched; every CTA then leaves at its next grid
// barrier.  A.dbg_trip makes every check of one site fail (its accesses are
// skipped), which exercises the reporting path without any bad index.  Without
// REXI_DEBUG both macros compile to the plain access.
#ifdef REXI_DEBUG
constexpr int kErrBounds = -7;          // REXI_EBOUNDS
__device__ double2 g_lz_sink[2];

__device__ __noinline__ void lz_fail(const LzArgs& A, int site, long long i, long long extent) {
    unsigned long long* r = reinterpret_cast<unsigned long long*>(A.dbg);
    if (r != nullptr) {
        if (atomicCAS(r, 0ull, (unsigned long long)site) == 0ull) {
            A.dbg[1] = i;
            A.dbg[2] = extent;
        }
        atomicAdd(r + 3, 1ull);
    }
    atomicExch(A.err, kErrBounds);
}
__device__ __forceinline__ bool lz_ok(const LzArgs& A, long long i, long long extent, int site) {
    if (i >= 0 && i < extent && site != A.dbg_trip) return true;
    lz_fail(A, site, i, extent);
    return false;
}
template <class T>
__device__ __forceinline__ T& lz_at(const LzArgs& A, T* base, long long i, long long extent, int site) {
    return lz_ok(A, i, extent, site) ? base[i] : *reinterpret_cast<T*>(g_lz_sink);
}
#define LZ_OK(i, extent, site) lz_ok(A, (long long)(i), (long long)(extent), (site))
#define LZ_AT(base, i, extent, site) lz_at(A, (base), (long long)(i), (long long)(extent), (site))

// Dynamic shared memory of the launch in bytes.
__device__ __forceinline__ unsigned dyn_bytes() {
    unsigned v;
    asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(v));
    return v;
}
#else
#define LZ_OK(i, extent, site) true
#define LZ_AT(base, i, extent, site) ((base)[i])
#endif

struct LzSmem {
    union {
        double2 coef[kLzMaxM];   // final pass: coefficients of the stored vectors
        float4 coefs[kLzMaxM];   //             resident mode: their hi/lo splits, scaled by 2^-E (r >= 1)
    };
    double2 c0;              //                            coefficient of the input state
    double cw, ca, cb;       // the update as applied: u_j = cw w' - ca u_{j-1} - cb u_{j-2}
    float cwf, caf[2], cbf[2];   // double-float recurrence: cw, ca, cb as (hi, lo) pairs (j == 2: cb in FP64)
    int cw_unit;             // cw == 1 (set with the coefficients: no FP64 compare per thread)
    float2 ry, rz;           // double-float recurrence: the stencil ratios r_y, r_z as pairs, and
    int uy, uz;              //   whether they are -1 (set once per launch)
    double n0;               // ||u_0||^2 of the substep
    double s_last, inv_s_last;   // scale s of the last update (u_{j-1} = s_{j-1} (...)), a power of two
    double hrho[2];          // rho = 1 / ||u|| of sweeps j-1, j-2 (from sweep 3 on: control CTA only)
    double hn[2];            // n = ||u||^2 of sweeps j-1, j-2 (idem)
    double ha[2], hsub[2], hsup[2];   // control CTA: T(i, i), T(i, i-1), T(i-1, i) for i = j-1, j-2
    double redd[kLzWarps][2];  // per-warp FP64 sums (sweep 0)
    float red[kLzWarps][4];  // per-warp double-float sums (n_hi, n_lo, p_hi, p_lo)
    float rprev_h, rprev_l;  // 1 / n_{j-1} in double-float
    float inv_sf_last;       // 1 / s_{j-1} (a power of two)
    int nring;               // resident mode: halo ring points of the tile
    int stop;
    int cexp;                // final pass, resident mode: largest biased exponent of the coefficients c_r, r >= 1
};

struct Tile {
    int x0, y0, z0;          // first interior point
    int tx, ty, tz;          // interior extent (ragged at the grid's edge)
    int ex, ey;              // extended extent in x and y (interior plus halo)
    int E, I;                // extended and interior point counts
};

__device__ __forceinline__ int wrapi(int x, int N) { return x < 0 ? x + N : (x >= N ? x - N : x); }

__device__ __forceinline__ Tile tile_of(const LzArgs& A, int t, int hx, int hy, int hz) {
    Tile T;
    const int ix = t % A.gx, r = t / A.gx, iy = r % A.gy, iz = r / A.gy;
    T.x0 = ix * A.tx;
    T.y0 = iy * A.ty;
    T.z0 = iz * A.tz;
    T.tx = min(A.tx, A.nx - T.x0);
    T.ty = min(A.ty, A.ny - T.y0);
    T.tz = min(A.tz, A.nz - T.z0);
    T.ex = T.tx + 2 * hx;
    T.ey = T.ty + 2 * hy;
    T.E = T.ex * T.ey * (T.tz + 2 * hz);
    T.I = T.tx * T.ty * T.tz;
    return T;
}

// u_r: u_0 is the substep's input state, u_1.. live in the basis.
__device__ __forceinline__ const double2* uvec(const LzArgs& A, const double2* u0, int r) {
    return r == 0 ? u0 : A.basis + (size_t)(r - 1) * (size_t)A.n;
}
__device__ __forceinline__ double2* uvec_w(const LzArgs& A, int r) {
    return A.basis + (size_t)(r - 1) * (size_t)A.n;
}

// acc + c u (complex), two fused multiply-adds per component.
__device__ __forceinline__ double2 cfma(double2 acc, double2 c, double2 u) {
    acc.x = fma(c.x, u.x, acc.x);
    acc.x = fma(-c.y, u.y, acc.x);
    acc.y = fma(c.x, u.y, acc.y);
    acc.y = fma(c.y, u.x, acc.y);
    return acc;
}
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 csc(double2 a, double s) { return make_double2(a.x * s, a.y * s); }

// Complex Givens rotation G = [c s; -conj(s) c] (c real) with G [x; h] = [r; 0]
// for complex x and real h >= 0; sabs = |s|; inv = 1 / r (0 when the column
// vanishes).
__device__ __forceinline__ void givens(double2 x, double h, double* c, double2* s, double* sabs, double2* r,
                                       double2* inv) {
    const double xx = x.x * x.x + x.y * x.y;
    if (h == 0.0) {
        *c = 1.0;
        *s = make_double2(0.0, 0.0);
        *sabs = 0.0;
        *r = x;
        const double rx = xx > 0.0 ? rsqrt(xx) : 0.0;
        *inv = make_double2(x.x * rx * rx, -x.y * rx * rx);
        return;
    }
    if (xx == 0.0) {
        *c = 0.0;
        *s = make_double2(1.0, 0.0);
        *sabs = 1.0;
        *r = make_double2(h, 0.0);
        const double rh = rsqrt(h * h);
        *inv = make_double2(rh, 0.0);
        return;
    }
    // two reciprocal square roots, no division
    const double rnx = rsqrt(xx), nu2 = fma(h, h, xx), rnu = rsqrt(nu2);
    const double2 ph = make_double2(x.x * rnx, x.y * rnx);
    *c = xx * rnx * rnu;
    *s = csc(ph, h * rnu);
    *sabs = fabs(h) * rnu;
    *r = csc(ph, nu2 * rnu);
    *inv = make_double2(ph.x * rnu, -ph.y * rnu);
}

__device__ __forceinline__ void trace_mark(const LzArgs& A, int code, int* tcount) {
    if (threadIdx.x == 0 && lz_bid(A) == 0) {
        const int c = *tcount;
        if (A.trace != nullptr && c < A.trace_cap) {
            A.trace[1 + 2 * c] = (unsigned long long)code;
            A.trace[2 + 2 * c] = global_ns();
            A.trace[0] = (unsigned long long)(c + 1);
        }
        *tcount = c + 1;
    }
}

// (h, l) += (bh, bl) in double-float: Knuth's two-sum of the leading parts,
// the trailing parts added to its error, renormalised.  Symmetric in its two
// operands, so butterfly reductions leave the same sum in every lane.
__device__ __forceinline__ void df_add(float& h, float& l, float bh, float bl) {
    const float s = __fadd_rn(h, bh);
    const float z = __fsub_rn(s, h);
    const float e = __fadd_rn(__fsub_rn(h, __fsub_rn(s, z)), __fsub_rn(bh, z));
    const float t = __fadd_rn(__fadd_rn(l, bl), e);
    h = __fadd_rn(s, t);
    l = __fsub_rn(t, __fsub_rn(h, s));
}

// Sum over the warp of the double-float pair (n, p) (butterfly: every lane
// ends with the same sums); FP32 pipe only.
__device__ __forceinline__ void warp_df_sum(float& nh, float& nl, float& ph, float& pl) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float a = __shfl_xor_sync(0xffffffffu, nh, o), b = __shfl_xor_sync(0xffffffffu, nl, o);
        const float c = __shfl_xor_sync(0xffffffffu, ph, o), d = __shfl_xor_sync(0xffffffffu, pl, o);
        df_add(nh, nl, a, b);
        df_add(ph, pl, c, d);
    }
}

// CTA sum of the pair; thread 0 receives (n_hi, n_lo, p_hi, p_lo).
__device__ __forceinline__ float4 cta_df_sum(LzSmem& sm, float nh, float nl, float ph, float pl) {
    warp_df_sum(nh, nl, ph, pl);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();                               // sm.red may still be read from the last sum
    if (lane == 0) {
        sm.red[warp][0] = nh;
        sm.red[warp][1] = nl;
        sm.red[warp][2] = ph;
        sm.red[warp][3] = pl;
    }
    __syncthreads();
    // the warps' sums: a butterfly over the first kLzWarps lanes of warp 0
    float4 t = make_float4(0.f, 0.f, 0.f, 0.f);
    if (warp == 0) {
        if (lane < kLzWarps) t = make_float4(sm.red[lane][0], sm.red[lane][1], sm.red[lane][2], sm.red[lane][3]);
#pragma unroll
        for (int o = kLzWarps / 2; o > 0; o >>= 1) {
            const float a = __shfl_xor_sync(0xffffffffu, t.x, o), b = __shfl_xor_sync(0xffffffffu, t.y, o);
            const float c = __shfl_xor_sync(0xffffffffu, t.z, o), d = __shfl_xor_sync(0xffffffffu, t.w, o);
            df_add(t.x, t.y, a, b);
            df_add(t.z, t.w, c, d);
        }
    }
    return t;
}

// Sweep 0 (u_0 = the caller's state, of any scale): the sums in FP64, CTA sum
// in a fixed order (thread 0 receives it), carried in the 16 bytes of a
// partial slot.
__device__ __forceinline__ double2 cta_f64_sum(LzSmem& sm, double n, double p) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        n += __shfl_xor_sync(0xffffffffu, n, o);
        p += __shfl_xor_sync(0xffffffffu, p, o);
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) {
        sm.redd[warp][0] = n;
        sm.redd[warp][1] = p;
    }
    __syncthreads();
    double2 t = make_double2(0.0, 0.0);
    if (threadIdx.x == 0)
        for (int w = 0; w < kLzWarps; ++w) {
            t.x += sm.redd[w][0];
            t.y += sm.redd[w][1];
        }
    return t;
}
__device__ __forceinline__ float4 pack_f64(double2 d) {
    return make_float4(__int_as_float(__double2loint(d.x)), __int_as_float(__double2hiint(d.x)),
                       __int_as_float(__double2loint(d.y)), __int_as_float(__double2hiint(d.y)));
}
__device__ __forceinline__ double2 unpack_f64(float4 f) {
    return make_double2(__hiloint2double(__float_as_int(f.y), __float_as_int(f.x)),
                        __hiloint2double(__float_as_int(f.w), __float_as_int(f.z)));
}

// Partials (||u||^2, Re u^H B u, each as a double-float pair) of sweep `par`
// of the tile CTAs (1..G-1): every thread loads its share (one round of loads,
// issued before the sweep's copies so they are not queued behind them) ...
struct PartLoad {
    float4 v[5];
};
__device__ __forceinline__ void load_partials(const LzArgs& A, int par, PartLoad& L) {
    const float4* p = A.part + (size_t)par * lz_nct(A);
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        const int c = 1 + threadIdx.x + q * kLzBlock;
        L.v[q] = c < lz_nct(A) && LZ_OK(par * lz_nct(A) + c, 2 * A.part_cap, LZ_SITE_PART)
                     ? __ldcg(p + c)
                     : make_float4(0.f, 0.f, 0.f, 0.f);
    }
}
// ... and the CTA sums them in double-float on the FP32 pipe (the FP64 pipe is
// busy with the co-resident CTA's sweep), in the same fixed order in every
// CTA; thread 0 receives the sums as FP64.
__device__ __forceinline__ float4 reduce_partials(const LzArgs& A, LzSmem& sm, int par, const PartLoad& L, bool f64) {
    if (f64) {
        // sweep 0: FP64 sums in the slots
        double n = 0.0, p = 0.0;
#pragma unroll
        for (int q = 0; q < 5; ++q) {
            const double2 d = unpack_f64(L.v[q]);
            n += d.x;
            p += d.y;
        }
        const float4* pp = A.part + (size_t)par * lz_nct(A);
        for (int c = 1 + threadIdx.x + 5 * kLzBlock; c < lz_nct(A); c += kLzBlock) {
            if (!LZ_OK(par * lz_nct(A) + c, 2 * A.part_cap, LZ_SITE_PART)) continue;
            const double2 d = unpack_f64(__ldcg(pp + c));
            n += d.x;
            p += d.y;
        }
        return pack_f64(cta_f64_sum(sm, n, p));
    }
    float nh = 0.f, nl = 0.f, ph = 0.f, pl = 0.f;
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        df_add(nh, nl, L.v[q].x, L.v[q].y);
        df_add(ph, pl, L.v[q].z, L.v[q].w);
    }
    const float4* p = A.part + (size_t)par * lz_nct(A);
    for (int c = 1 + threadIdx.x + 5 * kLzBlock; c < lz_nct(A); c += kLzBlock) {
        if (!LZ_OK(par * lz_nct(A) + c, 2 * A.part_cap, LZ_SITE_PART)) continue;
        const float4 w = __ldcg(p + c);
        df_add(nh, nl, w.x, w.y);
        df_add(ph, pl, w.z, w.w);
    }
    return cta_df_sum(sm, nh, nl, ph, pl);
}

// (h, l) = (ah + al)(bh + bl) in double-float (Dekker's product with a fused
// multiply-add, renormalised); about 2^-46 relative.
__device__ __forceinline__ void df_mul(float ah, float al, float bh, float bl, float& h, float& l) {
    const float p = __fmul_rn(ah, bh);
    float e = fmaf(ah, bh, -p);
    e = fmaf(ah, bl, e);
    e = fmaf(al, bh, e);
    h = __fadd_rn(p, e);
    l = __fsub_rn(e, __fsub_rn(h, p));
}
// (h, l) = 1 / (nh + nl) in double-float: one Newton step from the FP32 reciprocal.
__device__ __forceinline__ void df_recip(float nh, float nl, float& h, float& l) {
    const float r0 = __frcp_rn(nh);
    float e = fmaf(-nh, r0, 1.0f);
    e = fmaf(-nl, r0, e);
    const float c = __fmul_rn(r0, e);
    h = __fadd_rn(r0, c);
    l = __fsub_rn(c, __fsub_rn(h, r0));
}
// float -> double by integer operations (exact; subnormal floats become zero),
// so the scalar path of a Krylov step leaves the FP64 pipe to the sweeps.
__device__ __forceinline__ double f2d_int(float x) {
    const unsigned b = __float_as_uint(x);
    const unsigned sign = b & 0x80000000u, e = (b >> 23) & 0xFFu, m = b & 0x7FFFFFu;
    if (e == 0u) return __hiloint2double((int)sign, 0);
    const unsigned ex = e == 0xFFu ? 0x7FFu : e - 127u + 1023u;      // infinity and NaN stay so
    return __hiloint2double((int)(sign | (ex << 20) | (m >> 3)), (int)(m << 29));
}

// ---- asynchronous copies global -> shared (completion per thread) ---------
__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// ---- compensated (double-float) inner products on the FP32 pipe -------------
//
// The coefficients a_j, b_j and the norms set the local orthogonality of the
// basis; FP32 inner products leave components of relative size ~1e-7 (a wave
// packet that is an eigenvector then no longer breaks the recurrence down).
// Each FP64 operand is split into float hi + lo by integer operations only
// (48 of its 53 significand bits), products are formed exactly up to the lo*lo
// term (Dekker's product with a fused multiply-add) and summed with Knuth's
// two-sum; per-thread sums then continue in FP64.  Relative accuracy ~1e-13,
// without occupying the FP64 pipe.

// x ~= h + l with h the leading 24 significand bits (truncated) and l the next
// 24 (truncated); values below the float range become zero.
__device__ __forceinline__ void split_f64(double x, float* h, float* l) {
    const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
    const unsigned sign = hi & 0x80000000u;
    const int E = (int)((hi >> 20) & 0x7FFu);
    const int eh = E - 1023 + 127;
    if (eh <= 0 || eh >= 255) {
        *h = __uint_as_float(eh >= 255 ? (sign | 0x7F800000u) : sign);
        *l = __uint_as_float(sign);
        return;
    }
    *h = __uint_as_float(sign | ((unsigned)eh << 23) | ((hi & 0xFFFFFu) << 3) | (lo >> 29));
    const unsigned m = lo & 0x1FFFFFFFu;                  // the remaining 29 bits, unit 2^(E - 1075)
    const int k = 31 - __clz(m | 1u);                      // leading one of m (m = 0 handled below)
    const int el = k + E - 1075 + 127;
    if (m == 0u || el <= 0) {
        *l = __uint_as_float(sign);
        return;
    }
    const unsigned frac = k >= 23 ? (m >> (k - 23)) : (m << (23 - k));
    *l = __uint_as_float(sign | ((unsigned)el << 23) | (frac & 0x7FFFFFu));
}

// (sh, sl) += (ah + al)(bh + bl), dropping al*bl.
__device__ __forceinline__ void df_madd(float& sh, float& sl, float ah, float al, float bh, float bl) {
    const float p = __fmul_rn(ah, bh);
    float e = fmaf(ah, bh, -p);                            // exact rounding error of the product
    e = fmaf(ah, bl, e);
    e = fmaf(al, bh, e);
    const float t = __fadd_rn(sh, p);
    const float z = __fsub_rn(t, sh);
    const float err = __fadd_rn(__fsub_rn(sh, __fsub_rn(t, z)), __fsub_rn(p, z));
    sh = t;
    sl = __fadd_rn(sl, __fadd_rn(err, e));
}

constexpr int kCh = 4;          // points per thread whose loads are issued together

// Coordinates of the points e, e + kLzBlock, e + 2 kLzBlock, ... of a box
// (x fastest) kept incrementally: no division per point.
struct Walk {
    int x, y, z, dx, dy, dz;
    __device__ __forceinline__ void init(int e, int bx, int by) {
        x = e % bx;
        const int r = e / bx;
        y = r % by;
        z = r / by;
        dx = kLzBlock % bx;
        const int dr = kLzBlock / bx;
        dy = dr % by;
        dz = dr / by;
    }
    __device__ __forceinline__ void next(int bx, int by) {
        x += dx;
        y += dy;
        z += dz;
        if (x >= bx) {
            x -= bx;
            ++y;
        }
        if (y >= by) {
            y -= by;
            ++z;
        }
    }
};

// Global and extended index of the interior point at (x, y, z) of tile T.
__device__ __forceinline__ size_t int_index(const LzArgs& A, const Tile& T, const Walk& w, int hx, int hy, int hz,
                                            int* e) {
    *e = (w.x + hx) + T.ex * ((w.y + hy) + T.ey * (w.z + hz));
    return (size_t)(T.x0 + w.x) + (size_t)A.nx * ((size_t)(T.y0 + w.y) + (size_t)A.ny * (size_t)(T.z0 + w.z));
}

// Global index of the extended-box point at walk coordinates w of tile T
// (periodic wrap) and its interior index (-1 on the halo).
__device__ __forceinline__ size_t ext_index(const LzArgs& A, const Tile& T, const Walk& w, int hx, int hy, int hz,
                                            int* inner) {
    const int ix = w.x - hx, iy = w.y - hy, iz = w.z - hz;
    *inner = (ix >= 0 && ix < T.tx && iy >= 0 && iy < T.ty && iz >= 0 && iz < T.tz) ? ix + T.tx * (iy + T.ty * iz)
                                                                                   : -1;
    const int gxx = wrapi(T.x0 + ix, A.nx), gyy = wrapi(T.y0 + iy, A.ny), gzz = wrapi(T.z0 + iz, A.nz);
    return (size_t)gxx + (size_t)A.nx * ((size_t)gyy + (size_t)A.ny * (size_t)gzz);
}

// Shared memory of a tile CTA (all on the extended box of the tile, rows of
// T.ex points, except D, the diagonal on the interior):
//
//  streamed mode (a CTA with several tiles): every sweep stages the update's
//    inputs, W = B u_{j-1} (u_0 in sweep 0), U1 = u_{j-1}, U2 = u_{j-2}; W is
//    overwritten in place by u_j;
//  resident mode (one tile per CTA): the tile keeps its state between sweeps --
//    R[j mod 3] = u_j, u_{j-1}, u_{j-2} on the extended box (the halo values are
//    recomputed by this CTA exactly as the neighbours compute them), W = B u_{j-1}
//    (the interior from this CTA's own stencil), D loaded once.  A sweep needs
//    from the other CTAs only the halo ring of B u_{j-1}.
struct Stage {
    double2* W;
    double2* U1;       // streamed: u_{j-1}
    double2* U2;       // streamed: u_{j-2}
    double2* R0;       // resident: the last three vectors, R0 + k ext_max for k = 0, 1, 2
    int ext_max;       // points of the largest extended box and of the largest interior
    int int_max;
    double* D;
    int* ringE;        // resident: extended-box index and global index of every halo ring point
    int* ringG;
    __device__ __forceinline__ double2* R(int k) const { return R0 + (size_t)k * ext_max; }
};

// Streamed mode: issue the copies sweep j of tile t needs (one commit group).
__device__ void stage_tile(const LzArgs& A, const Stage& st, const double2* u0, int t, int j, int hx, int hy,
                           int hz) {
    const Tile T = tile_of(A, t, hx, hy, hz);
    const double2* wprev = A.wt + (size_t)((j - 1) & 1) * A.n;
    const double2* u1p = j >= 1 ? uvec(A, u0, j - 1) : nullptr;
    const double2* u2p = j >= 2 ? uvec(A, u0, j - 2) : nullptr;
    Walk w;
    w.init(threadIdx.x, T.ex, T.ey);
    for (int e = threadIdx.x; e < T.E; e += kLzBlock, w.next(T.ex, T.ey)) {
        int inner;
        const size_t g = ext_index(A, T, w, hx, hy, hz, &inner);
        if (!LZ_OK(e, st.ext_max, LZ_SITE_STAGE) || !LZ_OK(g, A.n, LZ_SITE_STAGE_SRC)) continue;
        if (j == 0) {
            cp_async16(st.W + e, u0 + g);
        } else {
            cp_async16(st.W + e, wprev + g);
            cp_async16(st.U1 + e, u1p + g);
            if (j >= 2) cp_async16(st.U2 + e, u2p + g);
        }
    }
    Walk wi;
    wi.init(threadIdx.x, T.tx, T.ty);
    for (int i = threadIdx.x; i < T.I; i += kLzBlock, wi.next(T.tx, T.ty)) {
        int e;
        const size_t g = int_index(A, T, wi, hx, hy, hz, &e);
        if (LZ_OK(i, st.int_max, LZ_SITE_STAGE) && LZ_OK(g, A.n, LZ_SITE_STAGE_SRC))
            cp_async8(st.D + i, A.df ? (const void*)(A.diag_df + g) : (const void*)(A.diag + g));
    }
    cp_async_commit();
}

// Resident mode: issue the copies of sweep j -- the extended box of u_0 in
// sweep 0, else the halo ring of B u_{j-1} (written by the neighbours).
__device__ void stage_resident(const LzArgs& A, const LzSmem& sm, const Stage& st, const double2* u0, int j, int hx,
                               int hy, int hz) {
    if (j == 0) {
        const Tile T = tile_of(A, lz_bid(A) - 1, hx, hy, hz);
        Walk w;
        w.init(threadIdx.x, T.ex, T.ey);
        for (int e = threadIdx.x; e < T.E; e += kLzBlock, w.next(T.ex, T.ey)) {
            int inner;
            const size_t g = ext_index(A, T, w, hx, hy, hz, &inner);
            if (LZ_OK(e, st.ext_max, LZ_SITE_STAGE) && LZ_OK(g, A.n, LZ_SITE_STAGE_SRC)) cp_async16(st.R(0) + e, u0 + g);
        }
    } else {
        const double2* wprev = A.wt + (size_t)((j - 1) & 1) * A.n;
        for (int q = threadIdx.x; q < sm.nring; q += kLzBlock) {
            if (!LZ_OK(q, st.ext_max - st.int_max, LZ_SITE_RING)) continue;
            const int e = st.ringE[q], g = st.ringG[q];
            if (LZ_OK(e, st.ext_max, LZ_SITE_STAGE) && LZ_OK(g, A.n, LZ_SITE_STAGE_SRC)) cp_async16(st.W + e, wprev + g);
        }
    }
    cp_async_commit();
}

// Resident mode, once per launch: the diagonal on the tile, and the list of
// the halo ring points (order immaterial: they are only copied).
__device__ void setup_resident(const LzArgs& A, LzSmem& sm, const Stage& st, int hx, int hy, int hz) {
    const Tile T = tile_of(A, lz_bid(A) - 1, hx, hy, hz);
    Walk wi;
    wi.init(threadIdx.x, T.tx, T.ty);
    for (int i = threadIdx.x; i < T.I; i += kLzBlock, wi.next(T.tx, T.ty)) {
        int e;
        const size_t g = int_index(A, T, wi, hx, hy, hz, &e);
        if (LZ_OK(i, st.int_max, LZ_SITE_STAGE) && LZ_OK(g, A.n, LZ_SITE_STAGE_SRC))
            cp_async8(st.D + i, A.df ? (const void*)(A.diag_df + g) : (const void*)(A.diag + g));
    }
    cp_async_commit();
    if (threadIdx.x == 0) sm.nring = 0;
    __syncthreads();
    Walk w;
    w.init(threadIdx.x, T.ex, T.ey);
    for (int e = threadIdx.x; e < T.E; e += kLzBlock, w.next(T.ex, T.ey)) {
        int inner;
        const size_t g = ext_index(A, T, w, hx, hy, hz, &inner);
        if (inner < 0) {
            const int q = atomicAdd(&sm.nring, 1);
            if (!LZ_OK(q, st.ext_max - st.int_max, LZ_SITE_RING)) continue;
            st.ringE[q] = e;
            st.ringG[q] = (int)g;
        }
    }
    __syncthreads();
}

// Phase A on one tile: v = rho (w - a u1 - b u2) on the extended box (in place
// of W in streamed mode, into R[j mod 3] in resident mode); with ujw given
// (streamed mode) the tile's own points are stored (they are u_j of the basis).
template <bool kUnit>
__device__ __forceinline__ void phase_a(const LzArgs& A, const Tile& T, const double2* W, const double2* U1,
                                        const double2* U2, double2* out, double2* ujw, int j, double cw, double ca,
                                        double cb, int hx, int hy, int hz) {
    Walk wa;
    wa.init(threadIdx.x, T.ex, T.ey);
    for (int e = threadIdx.x; e < T.E; e += kLzBlock, wa.next(T.ex, T.ey)) {
        const double2 w = W[e], u1 = U1[e];
        // kUnit: cw = 1, two fused multiply-adds per component
        double vx = fma(-ca, u1.x, kUnit ? w.x : cw * w.x), vy = fma(-ca, u1.y, kUnit ? w.y : cw * w.y);
        if (j >= 2) {
            const double2 u2 = U2[e];
            vx = fma(-cb, u2.x, vx);
            vy = fma(-cb, u2.y, vy);
        }
        const double2 v = make_double2(vx, vy);
        out[e] = v;
        const int ix = wa.x - hx, iy = wa.y - hy, iz = wa.z - hz;
        if (ujw != nullptr && ix >= 0 && ix < T.tx && iy >= 0 && iy < T.ty && iz >= 0 && iz < T.tz) {
            const size_t g =
                (size_t)(T.x0 + ix) + (size_t)A.nx * ((size_t)(T.y0 + iy) + (size_t)A.ny * (size_t)(T.z0 + iz));
            if (LZ_OK((long long)(j - 1) * A.n + (long long)g, (long long)(A.m + 2) * A.n, LZ_SITE_BASIS) &&
                LZ_OK(g, A.n, LZ_SITE_BASIS))
                ujw[g] = v;
        }
    }
}

// Phase B on one tile: B u_j from S (the extended box of u_j), stored to the
// global B u_j (and, resident mode, into Wown at the interior points); the
// compensated partial sums of ||u_j||^2 and Re u_j^H B u_j accumulate (kF64,
// sweep 0: FP64 sums, since u_0 may lie outside the FP32 range).  With
// ujs given (resident mode) u_j is stored to the basis as its hi/lo split
// (the pieces the inner products use): (re_hi, re_lo, im_hi, im_lo).
template <bool kF64>
__device__ __forceinline__ void phase_b(const LzArgs& A, const Tile& T, const double2* S, const double* D,
                                        const float2* Dd, double2* Wown, double2* wcur, float4* ujs, int hx, int hy,
                                        int hz, float& nh, float& nl, float& ph, float& pl, double& dn, double& dp) {
    // w' = B u / f with f = |a_d| of the first dimension the stencil reaches
    // (the a_d are negative): that dimension's neighbour pair enters with
    // weight -1 (one addition of negated operands), the others with r_d = a_d
    // / f, the diagonal (D = diag / f) with one fused multiply-add -- four FP64
    // operations per component in 2D
    const double ry = A.ratio[1], rz = A.ratio[2];
    const int sy = T.ex, sz = T.ex * T.ey;
    Walk wb;
    wb.init(threadIdx.x, T.tx, T.ty);
    for (int i = threadIdx.x; i < T.I; i += kLzBlock, wb.next(T.tx, T.ty)) {
        int e;
        const size_t g = int_index(A, T, wb, hx, hy, hz, &e);
        const double2 c = LZ_AT(S, e, T.E, LZ_SITE_STENCIL);
        double dg;
        if (kF64 && Dd != nullptr) {
            const float2 q = LZ_AT(Dd, i, T.I, LZ_SITE_STENCIL);      // double-float mode: the diagonal as pairs
            dg = (double)q.x + (double)q.y;
        } else {
            dg = LZ_AT(D, i, T.I, LZ_SITE_STENCIL);
        }
        double wx = 0.0, wy = 0.0;
        if (hx) {
            const double2 l = LZ_AT(S, e - 1, T.E, LZ_SITE_STENCIL), rr = LZ_AT(S, e + 1, T.E, LZ_SITE_STENCIL);
            wx = -l.x - rr.x;
            wy = -l.y - rr.y;
        }
        if (hy) {
            const double2 l = LZ_AT(S, e - sy, T.E, LZ_SITE_STENCIL), rr = LZ_AT(S, e + sy, T.E, LZ_SITE_STENCIL);
            if (hx) {
                wx = fma(ry, l.x + rr.x, wx);
                wy = fma(ry, l.y + rr.y, wy);
            } else {
                wx = -l.x - rr.x;
                wy = -l.y - rr.y;
            }
        }
        if (hz) {
            const double2 l = LZ_AT(S, e - sz, T.E, LZ_SITE_STENCIL), rr = LZ_AT(S, e + sz, T.E, LZ_SITE_STENCIL);
            if (hx || hy) {
                wx = fma(rz, l.x + rr.x, wx);
                wy = fma(rz, l.y + rr.y, wy);
            } else {
                wx = -l.x - rr.x;
                wy = -l.y - rr.y;
            }
        }
        wx = fma(dg, c.x, wx);
        wy = fma(dg, c.y, wy);
        const double2 wv = make_double2(wx, wy);
        if (LZ_OK(g, A.n, LZ_SITE_WT)) wcur[g] = wv;
        if (Wown) LZ_AT(Wown, e, T.E, LZ_SITE_STENCIL) = wv;
        if (kF64) {
            // sweep 0: u_0 at the caller's scale, the sums in FP64
            dn = fma(c.x, c.x, fma(c.y, c.y, dn));
            dp = fma(c.x, wx, fma(c.y, wy, dp));
            continue;
        }
        float cxh, cxl, cyh, cyl, wxh, wxl, wyh, wyl;
        split_f64(c.x, &cxh, &cxl);
        split_f64(c.y, &cyh, &cyl);
        if (ujs != nullptr && LZ_OK(g, A.n, LZ_SITE_BASIS)) ujs[g] = make_float4(cxh, cxl, cyh, cyl);
        split_f64(wx, &wxh, &wxl);
        split_f64(wy, &wyh, &wyl);
        df_madd(nh, nl, cxh, cxl, cxh, cxl);
        df_madd(nh, nl, cyh, cyl, cyh, cyl);
        df_madd(ph, pl, cxh, cxl, wxh, wxl);
        df_madd(ph, pl, cyh, cyl, wyh, wyl);
    }
}

// Sweep 0's phase B, kept out of line (it runs once per substep).
__device__ __noinline__ void phase_b_first(const LzArgs& A, const Tile& T, const double2* S, const double* D,
                                           double2* Wown, double2* wcur, int hx, int hy, int hz, double& dn,
                                           double& dp) {
    float nh = 0.f, nl = 0.f, ph = 0.f, pl = 0.f;
    const float2* Dd = A.df ? reinterpret_cast<const float2*>(D) : nullptr;
    phase_b<true>(A, T, S, D, Dd, Wown, wcur, nullptr, hx, hy, hz, nh, nl, ph, pl, dn, dp);
}

// ---- the recurrence in double-float (A.df) ----------------------------------
//
// From sweep 1 on, every vector of the recurrence (u_j on the extended box,
// w' = B u_j / f, the update's operands, the stored basis) is a pair of floats
// per component, (re_hi, re_lo, im_hi, im_lo) in one float4, and every
// operation runs on the FP32 pipe: the leading parts of a result's terms are
// summed by Knuth's two-sum (exactly), products are Dekker's (exact up to the
// lo*lo term, with a fused multiply-add), the trailing parts and the rounding
// errors are summed in FP32, and the pair is renormalised once per result.
// Each result is then within a few 2^-48 of the magnitude of its largest term:
// the error model of FP64 arithmetic with a unit roundoff 2^5 larger.  The
// recurrence's rounding enters psi' through the combined coefficients sum_k
// alpha_k y_k, not the individual weights, so its effect is that unit
// roundoff times sum_r |c_r| ||u_r|| (a few times 1e-14), far below the
// per-pole stopping tolerance.  Sweep 0 (the caller's state, at any scale)
// stays in FP64, sweep 1's update reads its FP64 results and rounds u_1 to
// pairs, and sweep 2 forms its u_0 term in FP64.

// (s, t) += x: two-sum of x into the leading sum s, its rounding error into t.
__device__ __forceinline__ void df_acc(float& s, float& t, float x) {
    const float r = __fadd_rn(s, x);
    const float z = __fsub_rn(r, s);
    t = __fadd_rn(t, __fadd_rn(__fsub_rn(s, __fsub_rn(r, z)), __fsub_rn(x, z)));
    s = r;
}
// (s, t) += (ah + al)(bh + bl): the rounded leading product into s, its exact
// error and the cross terms into t.
__device__ __forceinline__ void df_acc_mul(float& s, float& t, float ah, float al, float bh, float bl) {
    const float p = __fmul_rn(ah, bh);
    float e = fmaf(ah, bh, -p);
    e = fmaf(ah, bl, e);
    e = fmaf(al, bh, e);
    df_acc(s, t, p);
    t = __fadd_rn(t, e);
}
// (s, t) = (ah + al)(bh + bl), unnormalised.
__device__ __forceinline__ void df_start_mul(float& s, float& t, float ah, float al, float bh, float bl) {
    s = __fmul_rn(ah, bh);
    float e = fmaf(ah, bh, -s);
    e = fmaf(ah, bl, e);
    t = fmaf(al, bh, e);
}
// (s, t) -= (lh + ll) + (rh + rl): a neighbour pair of weight -1.
__device__ __forceinline__ void df_pair_unit(float& s, float& t, float lh, float ll, float rh, float rl) {
    df_acc(s, t, -lh);
    df_acc(s, t, -rh);
    t = __fsub_rn(__fsub_rn(t, ll), rl);
}
// (s, t) += r ((lh + ll) + (rh + rl)): a neighbour pair of weight r (a pair).
__device__ __forceinline__ void df_pair_ratio(float& s, float& t, float lh, float ll, float rh, float rl, float2 r) {
    float ph = 0.f, pl = 0.f;
    df_acc(ph, pl, lh);
    df_acc(ph, pl, rh);
    pl = __fadd_rn(pl, __fadd_rn(ll, rl));
    df_acc_mul(s, t, r.x, r.y, ph, pl);
}
// The pair s + t renormalised (h = fl(s + t), l = the rest).
__device__ __forceinline__ float2 df_norm(float s, float t) {
    const float h = __fadd_rn(s, t);
    return make_float2(h, __fsub_rn(t, __fsub_rn(h, s)));
}
// An FP64 value rounded to a pair (hi = fl32(x), lo = fl32(x - hi)).
__device__ __forceinline__ float2 df_from(double x) {
    const float h = __double2float_rn(x);
    return make_float2(h, __double2float_rn(x - (double)h));
}

// Sweep 1's update in double-float mode: v = cw w' - ca u_0 in FP64 from the
// FP64 results of sweep 0, rounded to pairs (into out; streamed mode: in
// place of W, and the tile's own points to ujw).
__device__ __noinline__ void phase_a_first_df(const LzArgs& A, const Tile& T, const double2* W, const double2* U1,
                                              float4* out, float4* ujw, double cw, double ca, int hx, int hy,
                                              int hz) {
    Walk wa;
    wa.init(threadIdx.x, T.ex, T.ey);
    for (int e = threadIdx.x; e < T.E; e += kLzBlock, wa.next(T.ex, T.ey)) {
        const double2 w = LZ_AT(W, e, T.E, LZ_SITE_STENCIL), u1 = LZ_AT(U1, e, T.E, LZ_SITE_STENCIL);
        const float2 vx = df_from(fma(-ca, u1.x, cw * w.x)), vy = df_from(fma(-ca, u1.y, cw * w.y));
        const float4 v = make_float4(vx.x, vx.y, vy.x, vy.y);
        LZ_AT(out, e, T.E, LZ_SITE_STENCIL) = v;
        const int ix = wa.x - hx, iy = wa.y - hy, iz = wa.z - hz;
        if (ujw != nullptr && ix >= 0 && ix < T.tx && iy >= 0 && iy < T.ty && iz >= 0 && iz < T.tz) {
            const size_t g =
                (size_t)(T.x0 + ix) + (size_t)A.nx * ((size_t)(T.y0 + iy) + (size_t)A.ny * (size_t)(T.z0 + iz));
            if (LZ_OK((long long)g, (long long)(A.m + 2) * A.n, LZ_SITE_BASIS) &&
                LZ_OK(g, A.n, LZ_SITE_BASIS))
                ujw[g] = v;
        }
    }
}

// Phase A in double-float mode, sweeps j >= 2: v = cw w' - ca u_{j-1} - cb
// u_{j-2} on the extended box (resident: into out = R[j mod 3]; streamed: in
// place of W, and the tile's own points to ujw).  kU0 (j = 2): u_{j-2} is the
// FP64 input state u_0, its term formed in FP64 with cb64 and rounded to pairs.
template <bool kUnit, bool kU0>
__device__ __forceinline__ void phase_a_df(const LzArgs& A, const Tile& Tr, const float4* __restrict__ W,
                                        const float4* __restrict__ U1, const void* U2, float4* out, float4* ujw, int j,
                                        float cw, float2 ca, float2 cb, double cb64, int hx, int hy, int hz) {
    // the tile and the grid extents in registers (a store of the loop could
    // alias a referenced object and force reloads)
    const Tile T = Tr;
    const size_t nx = (size_t)A.nx, nxy = (size_t)A.nx * (size_t)A.ny;
    Walk wa;
    wa.init(threadIdx.x, T.ex, T.ey);
    for (int e = threadIdx.x; e < T.E; e += kLzBlock, wa.next(T.ex, T.ey)) {
        const float4 w = LZ_AT(W, e, T.E, LZ_SITE_STENCIL), u1 = LZ_AT(U1, e, T.E, LZ_SITE_STENCIL);
        float xs = w.x, xt = w.y, ys = w.z, yt = w.w;
        if (!kUnit) {
            xs = __fmul_rn(cw, xs);
            xt = __fmul_rn(cw, xt);
            ys = __fmul_rn(cw, ys);
            yt = __fmul_rn(cw, yt);
        }
        df_acc_mul(xs, xt, -ca.x, -ca.y, u1.x, u1.y);
        df_acc_mul(ys, yt, -ca.x, -ca.y, u1.z, u1.w);
        if (kU0) {
            const double2 u2 = LZ_AT(reinterpret_cast<const double2*>(U2), e, T.E, LZ_SITE_STENCIL);
            const float2 px = df_from(-cb64 * u2.x), py = df_from(-cb64 * u2.y);
            df_acc(xs, xt, px.x);
            xt = __fadd_rn(xt, px.y);
            df_acc(ys, yt, py.x);
            yt = __fadd_rn(yt, py.y);
        } else {
            const float4 u2 = LZ_AT(reinterpret_cast<const float4*>(U2), e, T.E, LZ_SITE_STENCIL);
            df_acc_mul(xs, xt, -cb.x, -cb.y, u2.x, u2.y);
            df_acc_mul(ys, yt, -cb.x, -cb.y, u2.z, u2.w);
        }
        const float2 vx = df_norm(xs, xt), vy = df_norm(ys, yt);
        const float4 v = make_float4(vx.x, vx.y, vy.x, vy.y);
        LZ_AT(out, e, T.E, LZ_SITE_STENCIL) = v;
        const int ix = wa.x - hx, iy = wa.y - hy, iz = wa.z - hz;
        if (ujw != nullptr && ix >= 0 && ix < T.tx && iy >= 0 && iy < T.ty && iz >= 0 && iz < T.tz) {
            const size_t g = (size_t)(T.x0 + ix) + nx * (size_t)(T.y0 + iy) + nxy * (size_t)(T.z0 + iz);
            if (LZ_OK((long long)(j - 1) * A.n + (long long)g, (long long)(A.m + 2) * A.n, LZ_SITE_BASIS) &&
                LZ_OK(g, A.n, LZ_SITE_BASIS))
                ujw[g] = v;
        }
    }
}

// Phase B in double-float mode: w' = B u_j / f from S (u_j on the extended
// box, as pairs): the diagonal term, then the neighbour pairs (weight -1 for
// the first stencil dimension and wherever r_d = -1, as on a grid of equal
// spacings; else r_d as a pair); stored to the global B u_j and (resident
// mode) into Wown; u_j to the basis (ujs, resident mode); the compensated
// partial sums of ||u_j||^2 and Re u_j^H w' added to acc (n_hi, n_lo, p_hi,
// p_lo) and returned.  Out of line: its own register allocation (measured
// faster than inlined, and than two points per iteration).
__device__ __noinline__ float4 phase_b_df(const LzArgs& A, const Tile& Tr, const float4* __restrict__ S,
                                          const float2* __restrict__ D, float4* Wown, float4* wcur, float4* ujs,
                                          float2 ry, float2 rz, bool uy, bool uz, int hx, int hy, int hz,
                                          float4 acc) {
    // the tile, the grid extents and the sums in registers (a store of the
    // loop could alias a referenced object and force reloads)
    const Tile T = Tr;
    const size_t nx = (size_t)A.nx, nxy = (size_t)A.nx * (size_t)A.ny;
    float nh = acc.x, nl = acc.y, ph = acc.z, pl = acc.w;
    const int sy = T.ex, sz = T.ex * T.ey;
    Walk wb;
    wb.init(threadIdx.x, T.tx, T.ty);
    for (int i = threadIdx.x; i < T.I; i += kLzBlock, wb.next(T.tx, T.ty)) {
        const int e = (wb.x + hx) + T.ex * ((wb.y + hy) + T.ey * (wb.z + hz));
        const size_t g = (size_t)(T.x0 + wb.x) + nx * (size_t)(T.y0 + wb.y) + nxy * (size_t)(T.z0 + wb.z);
        const float4 c = LZ_AT(S, e, T.E, LZ_SITE_STENCIL);
        const float2 dg = LZ_AT(D, i, T.I, LZ_SITE_STENCIL);
        float xs, xt, ys, yt;
        df_start_mul(xs, xt, dg.x, dg.y, c.x, c.y);
        df_start_mul(ys, yt, dg.x, dg.y, c.z, c.w);
        if (hx) {
            const float4 l = LZ_AT(S, e - 1, T.E, LZ_SITE_STENCIL), r = LZ_AT(S, e + 1, T.E, LZ_SITE_STENCIL);
            df_pair_unit(xs, xt, l.x, l.y, r.x, r.y);
            df_pair_unit(ys, yt, l.z, l.w, r.z, r.w);
        }
        if (hy) {
            const float4 l = LZ_AT(S, e - sy, T.E, LZ_SITE_STENCIL), r = LZ_AT(S, e + sy, T.E, LZ_SITE_STENCIL);
            if (uy) {
                df_pair_unit(xs, xt, l.x, l.y, r.x, r.y);
                df_pair_unit(ys, yt, l.z, l.w, r.z, r.w);
            } else {
                df_pair_ratio(xs, xt, l.x, l.y, r.x, r.y, ry);
                df_pair_ratio(ys, yt, l.z, l.w, r.z, r.w, ry);
            }
        }
        if (hz) {
            const float4 l = LZ_AT(S, e - sz, T.E, LZ_SITE_STENCIL), r = LZ_AT(S, e + sz, T.E, LZ_SITE_STENCIL);
            if (uz) {
                df_pair_unit(xs, xt, l.x, l.y, r.x, r.y);
                df_pair_unit(ys, yt, l.z, l.w, r.z, r.w);
            } else {
                df_pair_ratio(xs, xt, l.x, l.y, r.x, r.y, rz);
                df_pair_ratio(ys, yt, l.z, l.w, r.z, r.w, rz);
            }
        }
        const float2 wx = df_norm(xs, xt), wy = df_norm(ys, yt);
        const float4 wv = make_float4(wx.x, wx.y, wy.x, wy.y);
        if (LZ_OK(g, A.n, LZ_SITE_WT)) wcur[g] = wv;
        if (Wown) LZ_AT(Wown, e, T.E, LZ_SITE_STENCIL) = wv;
        if (ujs != nullptr && LZ_OK(g, A.n, LZ_SITE_BASIS)) ujs[g] = c;
        df_madd(nh, nl, c.x, c.y, c.x, c.y);
        df_madd(nh, nl, c.z, c.w, c.z, c.w);
        df_madd(ph, pl, c.x, c.y, wv.x, wv.y);
        df_madd(ph, pl, c.z, c.w, wv.z, wv.w);
    }
    return make_float4(nh, nl, ph, pl);
}

// One Krylov sweep j over the tiles of this CTA (the first tile's copies were
// issued by the caller, and with `staged` already waited for and published by
// a barrier); part receives the CTA's partial sums (thread 0).
__device__ void sweep(const LzArgs& A, LzSmem& sm, const Stage& st, const double2* u0, int j, int hx, int hy, int hz,
                      bool staged, float4* part) {
    const int G1 = lz_nct(A) - 1;
    const double cw = sm.cw, ca = sm.ca, cb = sm.cb;
    double2* wcur = A.wt + (size_t)(j & 1) * A.n;
    double2* ujw = j >= 1 ? uvec_w(A, j) : nullptr;
    float nh = 0.f, nl = 0.f, ph = 0.f, pl = 0.f;
    double dn = 0.0, dp = 0.0;
    // double-float mode: the update's coefficients and the stencil ratios as
    // pairs, prepared in shared memory (an FP64 instruction per thread would
    // hold its SMSP's FP64 unit for about 64 cycles per warp)
    const bool df = A.df != 0;
    const bool unit = sm.cw_unit != 0;
    const float cwf = sm.cwf;
    const float2 caf = make_float2(sm.caf[0], sm.caf[1]), cbf = make_float2(sm.cbf[0], sm.cbf[1]);
    const float2 ry = sm.ry, rz = sm.rz;
    const bool uy = sm.uy != 0, uz = sm.uz != 0;
    if (A.resident) {
        if (lz_bid(A) - 1 < A.ntiles) {
            const Tile T = tile_of(A, lz_bid(A) - 1, hx, hy, hz);
            double2* S = st.R(j % 3);
            if (!staged) {
                cp_async_wait_all();
                __syncthreads();
            }
            const bool fits = LZ_OK(T.E, st.ext_max + 1, LZ_SITE_SMEM) && LZ_OK(T.I, st.int_max + 1, LZ_SITE_SMEM);
            if (fits && df) {
                float4* Sf = reinterpret_cast<float4*>(S);
                const float4* Wf = reinterpret_cast<const float4*>(st.W);
                if (j == 1) {
                    phase_a_first_df(A, T, st.W, st.R(0), Sf, nullptr, cw, ca, hx, hy, hz);
                } else if (j == 2) {
                    phase_a_df<false, true>(A, T, Wf, reinterpret_cast<const float4*>(st.R(1)), st.R(0), Sf, nullptr,
                                            j, cwf, caf, cbf, cb, hx, hy, hz);
                } else if (j >= 3) {
                    const float4* U1 = reinterpret_cast<const float4*>(st.R((j + 2) % 3));
                    const float4* U2 = reinterpret_cast<const float4*>(st.R((j + 1) % 3));
                    if (unit)
                        phase_a_df<true, false>(A, T, Wf, U1, U2, Sf, nullptr, j, cwf, caf, cbf, cb, hx, hy, hz);
                    else
                        phase_a_df<false, false>(A, T, Wf, U1, U2, Sf, nullptr, j, cwf, caf, cbf, cb, hx, hy, hz);
                }
                if (j >= 1) __syncthreads();
                float4* ujs = j >= 1 && LZ_OK(j - 1, A.m + 2, LZ_SITE_BASIS) ? reinterpret_cast<float4*>(ujw) : nullptr;
                if (j == 0) {
                    phase_b_first(A, T, S, st.D, st.W, wcur, hx, hy, hz, dn, dp);
                } else {
                    const float4 q = phase_b_df(A, T, Sf, reinterpret_cast<const float2*>(st.D),
                                                reinterpret_cast<float4*>(st.W), reinterpret_cast<float4*>(wcur), ujs,
                                                ry, rz, uy, uz, hx, hy, hz, make_float4(nh, nl, ph, pl));
                    nh = q.x;
                    nl = q.y;
                    ph = q.z;
                    pl = q.w;
                }
            } else if (fits) {
                if (j >= 1) {
                    if (unit)
                        phase_a<true>(A, T, st.W, st.R((j + 2) % 3), st.R((j + 1) % 3), S, nullptr, j, cw, ca, cb,
                                      hx, hy, hz);
                    else
                        phase_a<false>(A, T, st.W, st.R((j + 2) % 3), st.R((j + 1) % 3), S, nullptr, j, cw, ca, cb,
                                       hx, hy, hz);
                    __syncthreads();
                }
                float4* ujs = j >= 1 && LZ_OK(j - 1, A.m + 2, LZ_SITE_BASIS) ? reinterpret_cast<float4*>(ujw) : nullptr;
                if (j == 0)
                    phase_b_first(A, T, S, st.D, st.W, wcur, hx, hy, hz, dn, dp);
                else
                    phase_b<false>(A, T, S, st.D, nullptr, st.W, wcur, ujs, hx, hy, hz, nh, nl, ph, pl, dn, dp);
            }
        }
    } else {
        for (int t = lz_bid(A) - 1; t < A.ntiles; t += G1) {
            const bool first = t == lz_bid(A) - 1;
            if (!first) stage_tile(A, st, u0, t, j, hx, hy, hz);
            const Tile T = tile_of(A, t, hx, hy, hz);
            if (!(first && staged)) {
                cp_async_wait_all();
                __syncthreads();
            }
            if (!LZ_OK(T.E, st.ext_max + 1, LZ_SITE_SMEM) || !LZ_OK(T.I, st.int_max + 1, LZ_SITE_SMEM)) break;
            if (df) {
                // in place of W; the tile's own points of u_j to the basis
                float4* Wf = reinterpret_cast<float4*>(st.W);
                float4* ujf = reinterpret_cast<float4*>(ujw);
                if (j == 1) {
                    phase_a_first_df(A, T, st.W, st.U1, Wf, ujf, cw, ca, hx, hy, hz);
                } else if (j == 2) {
                    phase_a_df<false, true>(A, T, Wf, reinterpret_cast<const float4*>(st.U1), st.U2, Wf, ujf, j, cwf,
                                            caf, cbf, cb, hx, hy, hz);
                } else if (j >= 3) {
                    const float4* U1 = reinterpret_cast<const float4*>(st.U1);
                    const float4* U2 = reinterpret_cast<const float4*>(st.U2);
                    if (unit)
                        phase_a_df<true, false>(A, T, Wf, U1, U2, Wf, ujf, j, cwf, caf, cbf, cb, hx, hy, hz);
                    else
                        phase_a_df<false, false>(A, T, Wf, U1, U2, Wf, ujf, j, cwf, caf, cbf, cb, hx, hy, hz);
                }
                if (j >= 1) __syncthreads();
                if (j == 0) {
                    phase_b_first(A, T, st.W, st.D, nullptr, wcur, hx, hy, hz, dn, dp);
                } else {
                    const float4 q = phase_b_df(A, T, Wf, reinterpret_cast<const float2*>(st.D), nullptr,
                                                reinterpret_cast<float4*>(wcur), nullptr, ry, rz, uy, uz, hx, hy, hz,
                                                make_float4(nh, nl, ph, pl));
                    nh = q.x;
                    nl = q.y;
                    ph = q.z;
                    pl = q.w;
                }
                __syncthreads();                  // shared memory is restaged for the next tile
                continue;
            }
            if (j >= 1) {
                if (unit)
                    phase_a<true>(A, T, st.W, st.U1, st.U2, st.W, ujw, j, cw, ca, cb, hx, hy, hz);
                else
                    phase_a<false>(A, T, st.W, st.U1, st.U2, st.W, ujw, j, cw, ca, cb, hx, hy, hz);
                __syncthreads();
            }
            if (j == 0)
                phase_b_first(A, T, st.W, st.D, nullptr, wcur, hx, hy, hz, dn, dp);
            else
                phase_b<false>(A, T, st.W, st.D, nullptr, nullptr, wcur, nullptr, hx, hy, hz, nh, nl, ph, pl, dn, dp);
            __syncthreads();                      // shared memory is restaged for the next tile
        }
    }
    *part = j == 0 ? pack_f64(cta_f64_sum(sm, dn, dp)) : cta_df_sum(sm, nh, nl, ph, pl);
}

// Resident or double-float mode (the basis holds u_1, u_2, ... as pairs): the
// coefficients in sm.coef become c0 = c_0 (FP64, the input state's term) and,
// for r >= 1, the splits of 2^-E c_r with 2^E above the largest |Re|, |Im|, so
// the double-float products stay in the FP32 range; returns 2^E.
__device__ double split_coefficients(LzSmem& sm, int J) {
    if (threadIdx.x == 0) {
        sm.cexp = 0;
        sm.c0 = J >= 1 ? sm.coef[0] : make_double2(0.0, 0.0);
    }
    __syncthreads();
    double2 c[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const int r = threadIdx.x + q * kLzBlock;
        c[q] = r >= 1 && r < J ? sm.coef[r] : make_double2(0.0, 0.0);
        const int ex = (__double2hiint(c[q].x) >> 20) & 0x7FF, ey = (__double2hiint(c[q].y) >> 20) & 0x7FF;
        if (r >= 1 && r < J) atomicMax(&sm.cexp, max(ex, ey));
    }
    __syncthreads();
    // 2^-E with E = (largest biased exponent) - 1022: scaled values below one
    const int k = min(1000, max(-1000, 1022 - sm.cexp));
    const double down = __hiloint2double((1023 + k) << 20, 0);
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const int r = threadIdx.x + q * kLzBlock;
        if (r >= 1 && r < J) {
            float xh, xl, yh, yl;
            split_f64(c[q].x * down, &xh, &xl);
            split_f64(c[q].y * down, &yh, &yl);
            sm.coefs[r] = make_float4(xh, xl, yh, yl);
        }
    }
    __syncthreads();
    return __hiloint2double((1023 - k) << 20, 0);
}

// cp.async.wait_group with a run-time count (at most n groups pending).
__device__ __forceinline__ void cp_async_wait_upto(int n) {
    switch (n) {
        case 0: asm volatile("cp.async.wait_group 0;" ::: "memory"); break;
        case 1: asm volatile("cp.async.wait_group 1;" ::: "memory"); break;
        case 2: asm volatile("cp.async.wait_group 2;" ::: "memory"); break;
        case 3: asm volatile("cp.async.wait_group 3;" ::: "memory"); break;
        case 4: asm volatile("cp.async.wait_group 4;" ::: "memory"); break;
        case 5: asm volatile("cp.async.wait_group 5;" ::: "memory"); break;
        case 6: asm volatile("cp.async.wait_group 6;" ::: "memory"); break;
        default: asm volatile("cp.async.wait_group 7;" ::: "memory"); break;
    }
}

constexpr int kMaxDepth = 8;    // basis vectors a thread prefetches in the final pass

// Final pass over this CTA's tiles, dst = sum_{r < J} c_r u_r:
//  kSplit (resident or double-float mode; the basis holds u_1, u_2, ... as pairs):
//    dst = c_0 u_0 + 2^E sum_{1 <= r < J} (2^-E c_r) u_r, the sum in
//    double-float on the FP32 pipe (products exact up to the lo*lo term,
//    two-sum accumulation; about 2^-47 relative per term), the input state's
//    term and the scaling in FP64; sm.coefs holds the scaled splits;
//  else: FP64 complex multiply-adds with sm.coef.
// Every thread streams the basis entries of its own points through its own
// slots of the (then unused) dynamic shared memory by cp.async, `depth`
// vectors ahead, so depth * kCh loads per thread are in flight and no barrier
// is needed between a copy and its use (depth 0: plain loads).
template <bool kSplit>
__device__ void final_pass(const LzArgs& A, const LzSmem& sm, double up, const double2* u0, double2* dst, int J,
                           int hx, int hy, int hz, float4* slots, int depth) {
    const int G1 = lz_nct(A) - 1;
    const int rb = kSplit ? 1 : 0;                 // first vector through the slots
    for (int t = lz_bid(A) - 1; t < A.ntiles; t += G1) {
        const Tile T = tile_of(A, t, hx, hy, hz);
        Walk wb;
        wb.init(threadIdx.x, T.tx, T.ty);
        for (int i0 = threadIdx.x; i0 < T.I; i0 += kCh * kLzBlock) {
            size_t g[kCh];
            bool on[kCh];
#pragma unroll
            for (int q = 0; q < kCh; ++q) {
                int e;
                on[q] = i0 + q * kLzBlock < T.I;
                g[q] = 0;
                if (on[q]) {
                    g[q] = int_index(A, T, wb, hx, hy, hz, &e);
                    wb.next(T.tx, T.ty);
                    if (!LZ_OK(g[q], A.n, LZ_SITE_STATE)) on[q] = false;
                }
            }
            // the vectors newest first (the last ones written are the likeliest
            // still in L2): the k-th vector streamed is r = J - 1 - k
            const int nv = J - rb;
            // copies of the k-th vector into slot b (one commit group, possibly empty)
            auto issue = [&](int kv, int b) {
                const int r = J - 1 - kv;
                if (depth > 0 && kv < nv && LZ_OK(r, A.m + 3, LZ_SITE_BASIS)) {
                    const double2* u = uvec(A, u0, r);
#pragma unroll
                    for (int q = 0; q < kCh; ++q)
                        if (on[q]) cp_async16(slots + ((size_t)(b * kCh + q) * kLzBlock + threadIdx.x), u + g[q]);
                }
                cp_async_commit();
            };
            for (int b = 0; b + 1 < depth; ++b) issue(b, b);
            float rh[kCh], rl[kCh], ih[kCh], il[kCh];
            double2 acc[kCh];
#pragma unroll
            for (int q = 0; q < kCh; ++q) {
                rh[q] = rl[q] = ih[q] = il[q] = 0.f;
                acc[q] = make_double2(0.0, 0.0);
            }
            for (int k = 0; k < nv; ++k) {
                const int r = J - 1 - k;
                if (!LZ_OK(r, kLzMaxM, LZ_SITE_Y) || !LZ_OK(r, A.m + 3, LZ_SITE_BASIS)) break;
                int b = 0;
                if (depth > 0) {
                    issue(k + depth - 1, (k + depth - 1) % depth);
                    cp_async_wait_upto(depth - 1);
                    b = k % depth;
                }
                const double2* u = uvec(A, u0, r);
                if (kSplit) {
                    const float4 c = sm.coefs[r];
#pragma unroll
                    for (int q = 0; q < kCh; ++q) {
                        if (on[q]) {
                            const float4 v = depth > 0 ? slots[(size_t)(b * kCh + q) * kLzBlock + threadIdx.x]
                                                       : reinterpret_cast<const float4*>(u)[g[q]];
                            df_madd(rh[q], rl[q], c.x, c.y, v.x, v.y);      // Re c Re u
                            df_madd(rh[q], rl[q], -c.z, -c.w, v.z, v.w);    // - Im c Im u
                            df_madd(ih[q], il[q], c.x, c.y, v.z, v.w);      // Re c Im u
                            df_madd(ih[q], il[q], c.z, c.w, v.x, v.y);      // Im c Re u
                        }
                    }
                } else {
                    const double2 c = sm.coef[r];
#pragma unroll
                    for (int q = 0; q < kCh; ++q) {
                        if (on[q]) {
                            const double2 v = depth > 0 ? reinterpret_cast<const double2*>(
                                                              slots)[(size_t)(b * kCh + q) * kLzBlock + threadIdx.x]
                                                        : u[g[q]];
                            acc[q] = cfma(acc[q], c, v);
                        }
                    }
                }
            }
            cp_async_wait_all();
#pragma unroll
            for (int q = 0; q < kCh; ++q) {
                if (!on[q]) continue;
                if (kSplit) {
                    // (the pairs widened by integer operations: the FP64 unit
                    // takes only the multiply-adds)
                    const double2 a = cmul(sm.c0, u0[g[q]]);
                    dst[g[q]] = make_double2(fma(up, f2d_int(rh[q]), fma(up, f2d_int(rl[q]), a.x)),
                                             fma(up, f2d_int(ih[q]), fma(up, f2d_int(il[q]), a.y)));
                } else {
                    dst[g[q]] = acc[q];
                }
            }
        }
    }
}

// Per-pole state of the control CTA (thread k < K owns pole k).
struct PoleState {
    double c1, c2;           // rotations G_{c-1}, G_{c-2} (cosines)
    double2 s1, s2;          //                           (sines)
    double2 g;               // g_c, the right-hand side entry the next rotation acts on
    double2 g1, inv1;        // row c-1: g (final), 1 / R(c-1, c-1)
    double2 g2, inv2, r12;   // row c-2: g, 1 / R, R(c-2, c-1)
    double2 shift;
    int kk;                  // columns used (set when the pole stops)
    int done;                // 1 converged, 2 failed
    double bound;            // while the pole runs: L = ||z||_1 / |g| of the residual's coordinates
                             // (see pole_column); at the stop: the relative residual bound
};

// Row r of pole k's R, scaled by 1 / R(r, r), and its right-hand side entry:
// to the global rows and, for r < srows_cap, to the control CTA's shared
// memory (where the back substitution reads it without staging).
__device__ __forceinline__ void put_row(const LzArgs& A, int r, int k, double2 g, double2 inv, double2 r1, double2 r2,
                                        double2* srows, int srows_cap) {
    if (!LZ_OK(r, A.m, LZ_SITE_ROWS) || !LZ_OK(k, A.K, LZ_SITE_ROWS)) return;
    const double2 a = cmul(g, inv), b = cmul(r1, inv), c = cmul(r2, inv);
    double2* p = A.rows + ((size_t)r * A.K + k) * 3;
    p[0] = a;
    p[1] = b;
    p[2] = c;
    if (r < srows_cap) {
        double2* q = srows + ((size_t)r * A.K + k) * 3;
        q[0] = a;
        q[1] = b;
        q[2] = c;
    }
}

// Givens step of pole k on column c of T - s_k [I; 0]: entries up (row c-1),
// a_c - s_k (row c), lo (row c+1).  Returns true when the pole stops here.
__device__ bool pole_column(const LzArgs& A, PoleState& P, int k, int c, double up, double ac, double lo,
                            double tol_abs2, double2* srows, int srows_cap) {
    const double2 dg = make_double2(ac - P.shift.x, -P.shift.y);
    double2 xm1 = make_double2(up, 0.0);                   // row c-1 entry
    double2 r0 = make_double2(0.0, 0.0);                   // R(c-2, c)
    if (c >= 2) {
        r0 = csc(P.s2, up);
        xm1 = make_double2(P.c2 * up, 0.0);
    }
    double2 r1 = make_double2(0.0, 0.0);                   // R(c-1, c)
    double2 xc = dg;
    if (c >= 1) {
        r1 = cfma(csc(xm1, P.c1), P.s1, dg);
        const double2 cs1 = make_double2(-P.s1.x, P.s1.y);    // -conj(s1)
        xc = cfma(csc(dg, P.c1), cs1, xm1);
    }
    double c0, sa0;
    double2 s0, rcc, inv;
    givens(xc, lo, &c0, &s0, &sa0, &rcc, &inv);
    const double2 gc = csc(P.g, c0);
    const double2 gn = cmul(make_double2(-s0.x, s0.y), P.g);   // -conj(s0) g
    if (c >= 2) put_row(A, c - 2, k, P.g2, P.inv2, P.r12, r0, srows, srows_cap);
    // shift the pending rows and rotations
    P.g2 = P.g1;
    P.inv2 = P.inv1;
    P.r12 = r1;
    P.g1 = gc;
    P.inv1 = inv;
    P.c2 = P.c1;
    P.s2 = P.s1;
    P.c1 = c0;
    P.s1 = s0;
    P.g = gn;
    // The residual is Q_{c+2} z with z = G_0^H ... G_c^H (g_{c+1} e_{c+1}):
    // |z_{c+1}| = |g| c_c, |z_c| = |g| |s_c| c_{c-1}, |z_{c-1}| = |g| |s_c s_{c-1}|
    // c_{c-2}, ..., |z_0| = |g| |s_c ... s_0|, so with unit columns ||r|| <=
    // ||z||_1 = |g| L, L = c_c + |s_c| L_prev (L = 1 before column 0).  L never
    // exceeds sqrt(c + 2) (the bound for columns of unit norm without
    // orthogonality) and stays near c / (1 - |s|) while the pole converges.
    const double L = fma(sa0, P.bound, c0);
    P.bound = L;
    const double gg = gn.x * gn.x + gn.y * gn.y;
    if (gg * (L * L) <= tol_abs2) {
        // stop with c + 1 columns: rows c-1 and c complete with zeros
        const double2 z = make_double2(0.0, 0.0);
        if (c >= 1) put_row(A, c - 1, k, P.g2, P.inv2, P.r12, z, srows, srows_cap);
        put_row(A, c, k, P.g1, P.inv1, z, z, srows, srows_cap);
        P.kk = c + 1;
        P.done = 1;
        P.bound = sqrt(gg) * L;
        return true;
    }
    return false;
}

// Control CTA, as soon as every pole of the substep has stopped (J columns):
// y_k = R_k^{-1} g_k for every pole, then the coefficients of the final pass.  With
// J <= stage_rows the rows are already in shared memory (written there as they
// were formed) and y_k replaces each row's first entry; otherwise the rows are
// staged from global memory in chunks and y_k goes through global memory.
__device__ void control_finish(const LzArgs& A, LzSmem& sm, double2* stage, int stage_rows, PoleState& P, int J,
                               int s, double bnorm) {
    const int K = A.K;
    const int k = threadIdx.x;
    const bool inplace = J <= stage_rows;
    double2 y1 = make_double2(0.0, 0.0), y2 = make_double2(0.0, 0.0);
    for (int top = J; top > 0; top -= stage_rows) {
        const int lo = max(0, top - stage_rows);
        int cnt = (top - lo) * K * 3;
        if (!LZ_OK(cnt - 1, (long long)dyn_bytes() / sizeof(double2), LZ_SITE_ROWS) ||
            !LZ_OK((long long)top * K * 3 - 1, (long long)A.m * K * 3, LZ_SITE_ROWS))
            cnt = 0;
        __syncthreads();
        if (!inplace) {
#pragma unroll 8
            for (int q = threadIdx.x; q < cnt; q += kLzBlock) stage[q] = __ldcg(A.rows + (size_t)lo * K * 3 + q);
            __syncthreads();
        }
        if (k < K) {
            for (int r = top - 1; r >= lo; --r) {
                double2 y = make_double2(0.0, 0.0);
                double2* q = stage + ((size_t)(r - lo) * K + k) * 3;
                if (r < P.kk && cnt > 0) {
                    const double2 mr1 = make_double2(-q[1].x, -q[1].y), mr2 = make_double2(-q[2].x, -q[2].y);
                    y = cfma(cfma(q[0], mr2, y2), mr1, y1);
                }
                if (A.mode == LZ_STEP) {
                    if (inplace)
                        q[0] = y;
                    else if (LZ_OK((long long)r * K + k, (long long)A.m * K, LZ_SITE_Y))
                        A.ybuf[(size_t)r * K + k] = y;
                } else if (LZ_OK((long long)k * A.m + r, (long long)A.m * K, LZ_SITE_Y) &&
                           LZ_OK(r, A.m + 2, LZ_SITE_Y)) {
                    A.coef[(size_t)k * A.m + r] = csc(y, A.rho[r] * bnorm);
                }
                y2 = y1;
                y1 = y;
            }
        }
    }
    __syncthreads();
    if (A.mode == LZ_STEP) {
        // coef_r = ||psi|| rho_r sum_k alpha_k y_{k,r} (+ alpha_0 at r = 0): eight
        // threads per row, a fixed summation order
        const int q = threadIdx.x & 7;
        const int Jn = max(J, 1);
        for (int r0 = 0; r0 < Jn; r0 += kLzBlock / 8) {
            const int r = r0 + (threadIdx.x >> 3);
            double2 acc = make_double2(0.0, 0.0);
            if (r < J && LZ_OK((long long)r * K + K - 1, (long long)A.m * K, LZ_SITE_Y)) {
#pragma unroll 4
                for (int kq = q; kq < K; kq += 8)
                    acc = cfma(acc, __ldg(A.alpha + kq),
                               inplace ? stage[((size_t)r * K + kq) * 3] : A.ybuf[(size_t)r * K + kq]);
            }
#pragma unroll
            for (int o = 4; o > 0; o >>= 1) {
                acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
                acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
            }
            if (q == 0 && r < Jn && LZ_OK(r, A.m, LZ_SITE_Y) && LZ_OK(r, A.m + 2, LZ_SITE_Y)) {
                double2 c = r < J ? csc(acc, A.rho[r] * bnorm) : make_double2(0.0, 0.0);
                if (r == 0) {
                    c.x += A.alpha0.x;
                    c.y += A.alpha0.y;
                }
                A.coef[r] = c;
            }
        }
    }
    if (k < K) {
        ItemStats& st = A.stats[k];
        st.iters += P.kk;
        st.cycles += 1;
        st.iters_sq += P.kk * P.kk;
        st.max_sub_iters = max(st.max_sub_iters, P.kk);
        st.resid = fmax(st.resid, P.bound);
        if (P.done != 1) st.failed = 1;
    }
    if (threadIdx.x == 0 && LZ_OK(s, 2 * A.nsub, LZ_SITE_Y)) A.cols[s] = J;
    (void)sm;
}

// The launch's work for one problem, run by CTAs cta0 .. cta0 + ncta - 1.
__device__ __forceinline__ void lanczos_body(const LzArgs& A, double2* dyn, LzSmem& sm) {
    unsigned bar_gen = 0;                // grid barriers this CTA has passed (thread 0)
    const bool control = lz_bid(A) == 0;
    const bool has_tile = !control && lz_bid(A) - 1 < A.ntiles;
    const int hx = A.a[0] != 0.0 ? 1 : 0, hy = A.a[1] != 0.0 ? 1 : 0, hz = A.a[2] != 0.0 ? 1 : 0;
    const int ext_max = (A.tx + 2 * hx) * (A.ty + 2 * hy) * (A.tz + 2 * hz);
    Stage st;
    st.W = dyn;
    st.U1 = dyn + ext_max;
    st.U2 = dyn + 2 * ext_max;
    st.R0 = dyn + ext_max;
    st.ext_max = ext_max;
    st.D = (double*)(dyn + (A.resident ? 4 : 3) * ext_max);
    const int int_max = A.tx * A.ty * A.tz;
    st.int_max = int_max;
    st.ringE = (int*)(st.D + int_max);
    st.ringG = st.ringE + (ext_max - int_max);
    const int stage_rows = A.stage_rows;
    // final pass: the staging area (dead after the sweeps; the diagonal and the
    // ring list behind it stay) as prefetch slots of kCh * kLzBlock entries
    float4* slots = reinterpret_cast<float4*>(dyn);
    const int depth = min(kMaxDepth, (A.resident ? 4 : 3) * ext_max / (kCh * kLzBlock));
#ifdef REXI_DEBUG
    {
        // the layout above (tile CTAs) and the row staging (control CTA) fit the
        // launch's dynamic shared memory; the grid fits the partial-sum slots
        const long long need = control ? (long long)stage_rows * A.K * 3 * 16
                                       : (long long)(A.resident ? 4 : 3) * ext_max * 16 + (long long)int_max * 8 +
                                             (A.resident ? 8LL * (ext_max - int_max) : 0LL);
        if (!LZ_OK(need, (long long)dyn_bytes() + 1, LZ_SITE_SMEM) || !LZ_OK(lz_nct(A), A.part_cap + 1, LZ_SITE_PART))
            return;
    }
#endif
    if (threadIdx.x == 0) {
        sm.ry = df_from(A.ratio[1]);
        sm.rz = df_from(A.ratio[2]);
        sm.uy = A.ratio[1] == -1.0 ? 1 : 0;
        sm.uz = A.ratio[2] == -1.0 ? 1 : 0;
        sm.cw_unit = 1;
    }
    if (A.resident && !control) {
        if (has_tile) {
            setup_resident(A, sm, st, hx, hy, hz);
        } else {
            if (threadIdx.x == 0) sm.nring = 0;
            __syncthreads();
        }
    }
    int tcount = 0;
    trace_mark(A, 99, &tcount);
    PoleState P;
    for (int s = 0; s < A.nsub; ++s) {
        const double2* u0 = s == 0 ? A.in : ((s - 1) & 1 ? A.tmp1 : A.tmp0);
        double2* out = s == A.nsub - 1 ? A.out : (s & 1 ? A.tmp1 : A.tmp0);
        if (control && threadIdx.x < A.K) {
            P.c1 = P.c2 = 1.0;
            P.s1 = P.s2 = make_double2(0.0, 0.0);
            P.g = P.g1 = P.inv1 = P.g2 = P.inv2 = P.r12 = make_double2(0.0, 0.0);
            P.shift = A.shift[threadIdx.x];
            P.kk = 0;
            P.done = 0;
            P.bound = 1.0;                       // L before the first column
        }
        if (threadIdx.x == 0) {
            sm.n0 = 0.0;
            sm.s_last = sm.inv_s_last = 1.0;
            for (int q = 0; q < 2; ++q) sm.hrho[q] = sm.hn[q] = sm.ha[q] = sm.hsub[q] = sm.hsup[q] = 0.0;
            sm.rprev_h = sm.rprev_l = 0.f;
            sm.inv_sf_last = 1.0f;
        }
        __syncthreads();
        double tol_abs2 = 0.0, bnorm = 0.0;
        double upd_fl = 0.0;                           // FP64 flops per point of the updates (control CTA)
        int J = -1, sweeps = 0;
        for (int j = 0;; ++j) {
            // as the barrier opens: the partials and the stop word, then the
            // copies of this CTA's first tile
            PartLoad L;
            int stop_word = -1;
            if (j >= 1) {
                load_partials(A, (j - 1) & 1, L);
                if (threadIdx.x == 0 && LZ_OK(s, A.nsub, LZ_SITE_Y)) stop_word = __ldcg(A.stop + s);
            }
            if (has_tile) {
                if (A.resident)
                    stage_resident(A, sm, st, u0, j, hx, hy, hz);
                else
                    stage_tile(A, st, u0, lz_bid(A) - 1, j, hx, hy, hz);
            }
            if (j >= 1) {
                // coefficients of sweep j-1, the same in every CTA
                const float4 q = reduce_partials(A, sm, (j - 1) & 1, L, j == 1);
                if (threadIdx.x == 0) {
                    // sweep j-1 gave n = ||u_{j-1}||^2 and p = Re u_{j-1}^H w'
                    // (w' = B u_{j-1} / f).  The update is u_j = s_j (w' - alpha
                    // u_{j-1} - beta u_{j-2}) with alpha = p / n and beta = n /
                    // (s_{j-1} n_{j-2}); s_j = 1 (two fused multiply-adds per
                    // component) while n stays in [2^-30, 2^30], else the power of
                    // two that brings u_j back to unit scale.  With q_i = u_i / ||u_i||
                    // the columns of T follow from the coefficients as used:
                    // T(j-1, j-1) = f alpha, T(j-1, j-2) = f sqrt(n / n_{j-2}) /
                    // s_{j-1}, T(j-2, j-1) = f beta sqrt(n_{j-2} / n) (equal in exact
                    // arithmetic).  From sweep 2 on the tile CTAs form alpha and beta
                    // in double-float on the FP32 pipe (about 2^-46 relative; the
                    // control CTA takes T from the values actually used), so the
                    // step's scalar path costs two FP64 instructions.
                    double sj, inv_sj, ca, cb;
                    float rinv_h = 0.f, rinv_l = 0.f;          // 1 / n_{j-1} in double-float (j >= 3)
                    bool have_rinv = false;
                    if (j <= 2) {
                        // FP64: sweep 0's sums may lie outside the FP32 range, and
                        // beta at j = 2 divides by n_0
                        const double2 t = j == 1 ? unpack_f64(q)
                                                 : make_double2(f2d_int(q.x) + f2d_int(q.y), f2d_int(q.z) + f2d_int(q.w));
                        const double n = t.x;
                        const double rho = n > 0.0 ? rsqrt(n) : 0.0;
                        const double alpha = t.y * rho * rho;
                        const double rho2 = sm.hrho[0];
                        const double beta = j >= 2 ? n * rho2 * rho2 * sm.inv_s_last : 0.0;
                        sj = inv_sj = 1.0;
                        if (!A.unit_ok || !(n >= 0x1p-30 && n <= 0x1p30)) {
                            const int be = (__double2hiint(n) >> 20) & 0x7FF;
                            const int k = -((be - 1023) >> 1);           // s^2 n in [1/2, 4) for normal n
                            sj = __hiloint2double((1023 + k) << 20, 0);
                            inv_sj = __hiloint2double((1023 - k) << 20, 0);
                        }
                        ca = sj * alpha;
                        cb = sj * beta;
                        double alpha_used = alpha;
                        if (A.df && j == 2) {
                            // the pair the double-float update applies to u_1; T takes its value
                            const float2 pa = df_from(ca);
                            sm.caf[0] = pa.x;
                            sm.caf[1] = pa.y;
                            ca = (double)pa.x + (double)pa.y;
                            alpha_used = ca * inv_sj;
                        }
                        sm.cwf = __double2float_rn(sj);      // (used from j = 2 on: s_2 is within the FP32 range)
                        if (j == 1) sm.n0 = n;
                        sm.hrho[1] = sm.hrho[0];
                        sm.hrho[0] = rho;
                        sm.hn[1] = sm.hn[0];
                        sm.hn[0] = n;
                        if (control) {
                            const double sub = j >= 2 ? A.fold * n * rho * rho2 * sm.inv_s_last : 0.0;
                            sm.ha[1] = sm.ha[0];
                            sm.ha[0] = A.fold * alpha_used;
                            sm.hsub[1] = sm.hsub[0];
                            sm.hsub[0] = sub;
                            sm.hsup[1] = sm.hsup[0];
                            sm.hsup[0] = sub;
                            if (LZ_OK(j - 1, A.m + 2, LZ_SITE_Y)) A.rho[j - 1] = rho;
                        }
                    } else {
                        float sf = 1.0f, inv_sf = 1.0f;
                        sj = inv_sj = 1.0;
                        if (!A.unit_ok || !(q.x >= 0x1p-30f && q.x <= 0x1p30f)) {
                            const int be = (int)((__float_as_uint(q.x) >> 23) & 0xFFu);
                            const int k = -((be - 127) >> 1);
                            sf = __uint_as_float((unsigned)(127 + k) << 23);
                            inv_sf = __uint_as_float((unsigned)(127 - k) << 23);
                            sj = __hiloint2double((1023 + k) << 20, 0);
                            inv_sj = __hiloint2double((1023 - k) << 20, 0);
                        }
                        if (q.x > 0.f) df_recip(q.x, q.y, rinv_h, rinv_l);
                        have_rinv = true;
                        float ah, al, bh, bl;
                        df_mul(q.z, q.w, rinv_h, rinv_l, ah, al);             // alpha = p / n
                        df_mul(q.x, q.y, sm.rprev_h, sm.rprev_l, bh, bl);     // n / n_{j-2}
                        const float sb = __fmul_rn(sf, sm.inv_sf_last);        // s_j / s_{j-1}: a power of two
                        const float cah = __fmul_rn(ah, sf), cal = __fmul_rn(al, sf);
                        const float cbh = __fmul_rn(bh, sb), cbl = __fmul_rn(bl, sb);
                        // as doubles only where they are used: the FP64 update and the
                        // control CTA's columns of T (two FP64 instructions)
                        ca = cb = 0.0;
                        if (!A.df || control) {
                            ca = f2d_int(cah) + f2d_int(cal);
                            cb = f2d_int(cbh) + f2d_int(cbl);
                        }
                        // (the double-float update applies these pairs exactly)
                        sm.cwf = sf;
                        sm.caf[0] = cah;
                        sm.caf[1] = cal;
                        sm.cbf[0] = cbh;
                        sm.cbf[1] = cbl;
                        if (control) {
                            // the exact columns of T for these coefficients, in FP64
                            const double n = f2d_int(q.x) + f2d_int(q.y);
                            const double rho = n > 0.0 ? rsqrt(n) : 0.0;
                            const double rho2 = sm.hrho[0], n2 = sm.hn[0];
                            const double sub = A.fold * n * rho * rho2 * sm.inv_s_last;
                            sm.ha[1] = sm.ha[0];
                            sm.ha[0] = A.fold * (ca * inv_sj);
                            sm.hsub[1] = sm.hsub[0];
                            sm.hsub[0] = sub;
                            sm.hsup[1] = sm.hsup[0];
                            sm.hsup[0] = A.fold * (cb * inv_sj) * rho * (n2 * rho2);
                            sm.hrho[1] = sm.hrho[0];
                            sm.hrho[0] = rho;
                            sm.hn[1] = sm.hn[0];
                            sm.hn[0] = n;
                            if (LZ_OK(j - 1, A.m + 2, LZ_SITE_Y)) A.rho[j - 1] = rho;
                        }
                        sm.inv_sf_last = inv_sf;
                    }
                    if (j >= 2) {
                        // 1 / n_{j-1} for the next step's beta (n_{j-1} is in the FP32 range)
                        if (!have_rinv && q.x > 0.f) df_recip(q.x, q.y, rinv_h, rinv_l);
                        sm.rprev_h = rinv_h;
                        sm.rprev_l = rinv_l;
                    }
                    if (j <= 2) {
                        // (only j = 2's value is used, and s_2 is within the FP32 range)
                        const int k = min(126, max(-126, ((__double2hiint(sj) >> 20) & 0x7FF) - 1023));
                        sm.inv_sf_last = __uint_as_float((unsigned)(127 - k) << 23);
                    }
                    sm.cw = sj;
                    sm.cw_unit = sj == 1.0 ? 1 : 0;
                    sm.ca = ca;
                    sm.cb = cb;
                    sm.s_last = sj;
                    sm.inv_s_last = inv_sj;
                    sm.stop = stop_word;
                }
                // this barrier also publishes the first tile's copies to the sweep
                cp_async_wait_all();
                __syncthreads();
                if (sm.stop >= 0) {
                    J = sm.stop;
                    sweeps = j;                        // (no copy is in flight: waited above)
                    break;
                }
                if (j > A.m + 2) {                     // the control CTA stops by then: never taken
                    cp_async_wait_all();
                    if (threadIdx.x == 0) atomicExch(A.err, kErrInternal);
                    return;
                }
                // sweep j's update: a multiply and two (sweep 1: one) fused
                // multiply-adds per component, without the multiply when s = 1
                if (control && threadIdx.x == 0)
                    upd_fl += (sm.cw == 1.0 ? 0.0 : 2.0) + (j == 1 ? 4.0 : 8.0);
            }
            if (!control) {
                float4 part;
                sweep(A, sm, st, u0, j, hx, hy, hz, j >= 1, &part);
                if (threadIdx.x == 0 && LZ_OK((j & 1) * lz_nct(A) + lz_bid(A), 2 * A.part_cap, LZ_SITE_PART))
                    A.part[(size_t)(j & 1) * lz_nct(A) + lz_bid(A)] = part;
            } else if (j >= 1) {
                // the control CTA works one column behind: column c = j - 2 is
                // complete once the norm of u_{j-1} (its subdiagonal) is known
                int stop_now = -1;                     // the substep's column count, once known
                if (j == 1) {
                    const double n0 = sm.n0;
                    // the poles solve for psi / ||psi|| (right-hand side e_1, for
                    // any scale of psi); ||psi|| enters the final coefficients
                    bnorm = sqrt(n0);
                    const double ta = A.tol / 1.0001;
                    tol_abs2 = ta * ta;
                    if (threadIdx.x < A.K) P.g = make_double2(1.0, 0.0);
                    // a zero state needs no columns; a non-finite one fails every pole
                    if (!(n0 > 0.0 && n0 <= 1.0e300)) stop_now = 0;
                    if (threadIdx.x < A.K && !(n0 > 0.0)) P.done = n0 == 0.0 ? 1 : 2;
                    if (threadIdx.x < A.K && !(n0 <= 1.0e300)) P.done = 2;
                    if (threadIdx.x < A.K && P.done != 0) P.bound = 0.0;   // no columns: no residual bound
                } else {
                    const int c = j - 2;
                    // T[c-1, c] = T[c, c-1] and T[c+1, c], from the last two reductions
                    const double up = c >= 1 ? sm.hsup[1] : 0.0;
                    const double lo = sm.hsub[0];
                    const double ac = sm.ha[1];
                    int active = 0;
                    if (threadIdx.x < A.K && P.done == 0) {
                        pole_column(A, P, threadIdx.x, c, up, ac, lo, tol_abs2, dyn, stage_rows);
                        if (P.done == 0 && c + 1 >= A.m) {
                            P.done = 2;
                            P.kk = c + 1;
                            const double gg = P.g.x * P.g.x + P.g.y * P.g.y;
                            P.bound = sqrt(gg) * P.bound;
                            const double2 z = make_double2(0.0, 0.0);
                            if (c >= 1) put_row(A, c - 1, threadIdx.x, P.g2, P.inv2, P.r12, z, dyn, stage_rows);
                            put_row(A, c, threadIdx.x, P.g1, P.inv1, z, z, dyn, stage_rows);
                        }
                        active = P.done == 0;
                    }
                    const int still = __syncthreads_count(active);
                    if (still == 0) stop_now = c + 1;
                }
                if (stop_now >= 0) {
                    // every pole has stopped: publish the column count and form
                    // y_k and the coefficients of the final pass now, while the
                    // tile CTAs run the sweep whose result is not needed (the
                    // barrier below waits for it; the one after the loop then
                    // opens at once)
                    if (threadIdx.x == 0) __stcg(A.stop + s, stop_now);
                    control_finish(A, sm, dyn, stage_rows, P, stop_now, s, bnorm);
                }
            }
            if (!grid_sync(A.bar, (unsigned)A.ncta, bar_gen, A.err, A.timeout_ns)) return;
            trace_mark(A, TR_LZ_SWEEP, &tcount);
        }
        // (the control CTA formed y_k and the coefficients as the poles stopped)
        if (!grid_sync(A.bar, (unsigned)A.ncta, bar_gen, A.err, A.timeout_ns)) return;
        trace_mark(A, TR_LZ_SOLVE, &tcount);
        if (control && threadIdx.x == 0) {
            // (the control CTA is idle during the final pass)
            if (LZ_OK(A.nsub + s, 2 * A.nsub, LZ_SITE_Y)) A.cols[A.nsub + s] = sweeps;
            // the work the specified recurrence moves and computes (halo
            // re-reads not counted): sweep 0 reads u_0 and the diagonal and
            // writes B u_0; sweep 1 also reads B u_0 and writes u_1; later
            // sweeps read B u_{j-1}, u_{j-1}, u_{j-2} and write u_j, B u_j
            const double n = (double)A.n;
            const int d = hx + hy + hz;
            const double later = (double)max(sweeps - 2, 0);
            double by = (sweeps >= 1 ? 40.0 : 0.0) + (sweeps >= 2 ? 72.0 : 0.0) + 88.0 * later;
            // (double-float mode: FP64 work in sweep 0's stencil, sweep 1's
            // update and sweep 2's u_0 term only)
            double fl = A.df ? 6.0 * d * min(sweeps, 1) + (sweeps >= 2 ? 4.0 : 0.0) + (sweeps >= 3 ? 2.0 : 0.0)
                             : 6.0 * d * sweeps + upd_fl;
            // the final pass reads J vectors and writes one output per pole set;
            // its FP64 work: a complex multiply-add per vector, or (resident
            // mode, the sum in double-float on the FP32 pipe) the input
            // state's term and the scaling
            const int Jn = A.mode == LZ_STEP ? max(J, 1) : J;
            const int outs = A.mode == LZ_STEP ? 1 : A.K;
            by += outs * 16.0 * (Jn + 1);
            fl += outs * (A.resident || A.df ? 12.0 : 8.0 * Jn);
            // FP32-pipe arithmetic, as the code issues it: the compensated
            // inner products of sweeps >= 1 (four Dekker multiply-adds of 12
            // operations per point); double-float mode: also the stencil (per
            // component a product of 4, a neighbour pair of weight -1: 14, a
            // pair of weight r_d: 25, a renormalisation: 3) and the update of
            // sweeps >= 2 (per component two multiply-adds of 11 and a
            // renormalisation); the final pass in double-float (resident or
            // double-float mode): four multiply-adds per vector u_1, u_2, ...
            double ops = 48.0 * max(sweeps - 1, 0);
            if (A.df) {
                double pairs = 0.0;
                for (int q = 0; q < 3; ++q)
                    if ((q == 0 && hx) || (q == 1 && hy) || (q == 2 && hz))
                        pairs += (q == 0 || A.ratio[q] == -1.0) ? 14.0 : 25.0;
                ops += 2.0 * (7.0 + pairs) * max(sweeps - 1, 0) + 50.0 * max(sweeps - 2, 0);
            }
            if (A.resident || A.df) ops += outs * 48.0 * max(Jn - 1, 0);
            if (A.bytes != nullptr) {
                A.bytes[0] += (unsigned long long)(by * n);
                A.bytes[1] += (unsigned long long)(fl * n);
                A.bytes[2] += (unsigned long long)(ops * n);
            }
        }
        if (!control) {
            if (A.mode == LZ_STEP) {
                const int Jn = max(J, 1);
                for (int r = threadIdx.x; r < Jn; r += kLzBlock)
                    if (LZ_OK(r, kLzMaxM, LZ_SITE_Y) && LZ_OK(r, A.m, LZ_SITE_Y)) sm.coef[r] = __ldcg(A.coef + r);
                __syncthreads();
                if (A.resident || A.df)
                    final_pass<true>(A, sm, split_coefficients(sm, Jn), u0, out, Jn, hx, hy, hz, slots, depth);
                else
                    final_pass<false>(A, sm, 1.0, u0, out, Jn, hx, hy, hz, slots, depth);
            } else {
                for (int k = 0; k < A.K; ++k) {
                    __syncthreads();
                    for (int r = threadIdx.x; r < J; r += kLzBlock)
                        if (LZ_OK(r, kLzMaxM, LZ_SITE_Y) && LZ_OK(r, A.m, LZ_SITE_Y))
                            sm.coef[r] = __ldcg(A.coef + (size_t)k * A.m + r);
                    __syncthreads();
                    double2* xk = A.out + (size_t)k * A.n;
                    if (A.resident || A.df)
                        final_pass<true>(A, sm, split_coefficients(sm, J), u0, xk, J, hx, hy, hz, slots, depth);
                    else
                        final_pass<false>(A, sm, 1.0, u0, xk, J, hx, hy, hz, slots, depth);
                }
            }
        }
        if (s + 1 < A.nsub) {
            if (!grid_sync(A.bar, (unsigned)A.ncta, bar_gen, A.err, A.timeout_ns)) return;
            trace_mark(A, TR_LZ_SUM, &tcount);
        }
    }
}

__global__ void __launch_bounds__(kLzBlock, 2) lanczos_kernel(const __grid_constant__ LzArgs A) {
    extern __shared__ double2 dyn[];
    __shared__ LzSmem sm;
    lanczos_body(A, dyn, sm);
}

// Several problems in one launch: CTA c works for problem cta_prob[c], whose
// descriptor (with the call's input and output states) it copies to shared
// memory; each problem's CTAs synchronise only among themselves.
__global__ void __launch_bounds__(kLzBlock, 2)
    lanczos_batched_kernel(const LzArgs* __restrict__ args, const unsigned char* __restrict__ cta_prob,
                           const __grid_constant__ LzIO io) {
    extern __shared__ double2 dyn[];
    __shared__ LzSmem sm;
    __shared__ LzArgs a;
    if (threadIdx.x == 0) {
        const int p = cta_prob[blockIdx.x];
        a = args[p];
        a.in = io.in[p];
        a.out = io.out[p];
    }
    __syncthreads();
    lanczos_body(a, dyn, sm);
}

// Before a batched launch: every problem's barrier, error, work counters,
// statistics and stop words (block p: problem p).
__global__ void lanczos_reset_kernel(const LzArgs* __restrict__ args) {
    const LzArgs& A = args[blockIdx.x];
    if (threadIdx.x < 3) A.bar[threadIdx.x] = 0u;
    if (threadIdx.x == 0) *A.err = 0;
    if (threadIdx.x < 3 && A.bytes != nullptr) A.bytes[threadIdx.x] = 0ull;
    if (threadIdx.x < 4 && A.dbg != nullptr) A.dbg[threadIdx.x] = 0;
    int* st = reinterpret_cast<int*>(A.stats);
    const int words = (int)(A.K * sizeof(ItemStats) / sizeof(int));
    for (int q = threadIdx.x; q < words; q += blockDim.x) st[q] = 0;
    for (int q = threadIdx.x; q < A.nsub; q += blockDim.x) A.stop[q] = -1;
}

}  // namespace

size_t lanczos_smem_bytes(int tx, int ty, int tz, int hx, int hy, int hz, bool resident) {
    const size_t ext = (size_t)(tx + 2 * hx) * (ty + 2 * hy) * (tz + 2 * hz);
    const size_t inner = (size_t)tx * ty * tz;
    return (resident ? 4 : 3) * ext * sizeof(double2) + inner * sizeof(double) +
           (resident ? 2 * (ext - inner) * sizeof(int) : 0);
}

size_t lanczos_static_smem() {
    cudaFuncAttributes fa, fb;
    if (cudaFuncGetAttributes(&fa, lanczos_kernel) != cudaSuccess ||
        cudaFuncGetAttributes(&fb, lanczos_batched_kernel) != cudaSuccess)
        return 0;
    return std::max(fa.sharedSizeBytes, fb.sharedSizeBytes);
}

int lanczos_max_grid(size_t smem, int device, bool batched) {
    int per_sm = 0, sms = 0;
    const void* k = batched ? (const void*)lanczos_batched_kernel : (const void*)lanczos_kernel;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return -1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kLzBlock, smem) != cudaSuccess) return -1;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return -1;
    return per_sm * sms;
}

cudaError_t launch_lanczos(const LzArgs& args, int grid, size_t smem, cudaStream_t stream) {
    cudaError_t e = cudaFuncSetAttribute(lanczos_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    void* params[] = {(void*)&args};
    return cudaLaunchCooperativeKernel((const void*)lanczos_kernel, dim3(grid), dim3(kLzBlock), params, smem, stream);
}

cudaError_t lanczos_reset(const LzArgs* d_args, int B, cudaStream_t stream) {
    lanczos_reset_kernel<<<B, 128, 0, stream>>>(d_args);
    return cudaGetLastError();
}

cudaError_t launch_lanczos_batched(const LzArgs* d_args, const unsigned char* d_cta_prob, const LzIO& io, int grid,
                                   size_t smem, cudaStream_t stream) {
    cudaError_t e =
        cudaFuncSetAttribute(lanczos_batched_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    void* params[] = {(void*)&d_args, (void*)&d_cta_prob, (void*)&io};
    return cudaLaunchCooperativeKernel((const void*)lanczos_batched_kernel, dim3(grid), dim3(kLzBlock), params, smem,
                                       stream);
}

}  // namespace rexi
