// Persistent REXI engine for sm_103a.
//
// One cooperative launch runs a whole call: n_sub substeps of Eq. (5) of
// Rittich & Speck (arXiv:1912.03312), each made of K independent restarted
// GMRES solves of (tau H - z_k I) x_k = b (Sec. 3.1: the K systems are
// independent tasks) followed by the weighted pole sum.  All solves of all
// problems advance in lock step through grid-wide phases separated by bounded
// grid barriers:
//
//   E3  residual   r = b - A x in FP64 (x = 0 on the first cycle), stored as u_0
//   E4  decide     per item: converged / failed / start a cycle with s_0 = 1/||r||
//   P1  matvec     w = A (s_j u_j) (stencil, fused diagonal shift), p1 = U_j^H w
//   P2  CGS pass 2 p2 = U_j^H (w - V_j h1)
//   P3  update     w <- w - V_j (h1 + h2), ||w||^2                (CGS2)
//   P4  Givens     per item: rotate the Hessenberg column, update |g_{j+1}|
//   E2  update     x += V_k y, y = R^{-1} g                      (FP64 accumulation)
//   PS  pole sum   psi' = alpha_0 b + sum_k alpha_k x_k          (FP64)
//   BA  adjoint    G' = conj(alpha_0) G + sum conj(alpha_k) Y_k,
//                  dL/dV -= tau Re sum alpha_k conj(Y_k) X_k
//
// A "phase" is the flat list of (item, tile) tasks of the items in the right
// state, split evenly over the CTAs.  Partial dot products are written per run
// and reduced (FP64 for CGS2, FP32 for the one-reduction Arnoldi) by the CTAs
// of the next phase.  Basis vectors u_i are stored unnormalised; the column is
// s_i u_i with an FP64 scale s_i.
#include <algorithm>
#include <cstdint>

#include "engine.h"

namespace rexi {

namespace {

constexpr int kWarps = kBlock / 32;
constexpr int kErrTimeout = -5;   // REXI_ETIMEOUT

template <typename T> struct C2;
template <> struct C2<float> { typedef float2 t; };
template <> struct C2<double> { typedef double2 t; };

__device__ __forceinline__ float2 mk2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ double2 mk2(double a, double b) { return make_double2(a, b); }

template <typename V> __device__ __forceinline__ V cvt2(double2 a);
template <> __device__ __forceinline__ float2 cvt2<float2>(double2 a) {
    return make_float2((float)a.x, (float)a.y);
}
template <> __device__ __forceinline__ double2 cvt2<double2>(double2 a) { return a; }
__device__ __forceinline__ double2 up2(float2 a) { return make_double2(a.x, a.y); }
__device__ __forceinline__ double2 up2(double2 a) { return a; }

// Double to float by integer operations only (rounding toward zero; results
// below the float range become signed zero, above it (and NaN) signed
// infinity), so the conversion does not occupy the FP64 pipe.
__device__ __forceinline__ float f64_to_f32_rz(double x) {
    const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
    const unsigned sign = hi & 0x80000000u;
    const int e = (int)((hi >> 20) & 0x7FFu) - 1023 + 127;
    if (e <= 0) return __uint_as_float(sign);
    if (e >= 255) return __uint_as_float(sign | 0x7F800000u);
    return __uint_as_float(sign | ((unsigned)e << 23) | ((hi & 0xFFFFFu) << 3) | (lo >> 29));
}
__device__ __forceinline__ float2 dot_f2(double2 a) { return make_float2(f64_to_f32_rz(a.x), f64_to_f32_rz(a.y)); }
__device__ __forceinline__ float2 dot_f2(float2 a) { return a; }

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }

// acc + c u and acc - c u as chains of fused multiply-adds, two per component
// (written out so that no separate multiply or add is left over: the FP64
// pipe is the scarce unit of the sweeps).
__device__ __forceinline__ float fmat(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fmat(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ double2 cfma(double2 acc, double2 c, double2 u) {
    return make_double2(fma(-c.y, u.y, fma(c.x, u.x, acc.x)), fma(c.y, u.x, fma(c.x, u.y, acc.y)));
}
__device__ __forceinline__ double2 cfms(double2 acc, double2 c, double2 u) {
    return make_double2(fma(c.y, u.y, fma(-c.x, u.x, acc.x)), fma(-c.y, u.x, fma(-c.x, u.y, acc.y)));
}
__device__ __forceinline__ float2 cfma(float2 acc, float2 c, float2 u) {
    return make_float2(fmaf(-c.y, u.y, fmaf(c.x, u.x, acc.x)), fmaf(c.y, u.x, fmaf(c.x, u.y, acc.y)));
}
__device__ __forceinline__ float2 cfms(float2 acc, float2 c, float2 u) {
    return make_float2(fmaf(c.y, u.y, fmaf(-c.x, u.x, acc.x)), fmaf(-c.y, u.x, fmaf(-c.x, u.y, acc.y)));
}

// State words, Hessenberg columns and partial sums written inside this launch
// are loaded through L2 only (.cg).
//
// Vector data (basis vectors, w, x, the step states) is loaded with plain
// loads, which may be served by L1: every read of such data is separated from
// the stores it depends on by a grid barrier (fence and arrival by each CTA,
// release by the completing one, ld.acquire.gpu by each waiting CTA, then a
// CTA barrier), so by the PTX memory model the load observes those stores
// whatever the cache operator.
// The stencil's neighbour loads then mostly hit the lines of the CTA's own
// centre loads.
__device__ __forceinline__ float2 ldv(const float2* p) { return *p; }
__device__ __forceinline__ double2 ldv(const double2* p) { return *p; }
__device__ __forceinline__ float2 ldp(const float2* p) { return __ldcg(p); }
__device__ __forceinline__ double2 ldp(const double2* p) { return __ldcg(p); }
__device__ __forceinline__ double ldd(const double* p) { return __ldcg(p); }
__device__ __forceinline__ int ldi(const int* p) { return __ldcg(p); }

template <typename V> __device__ __forceinline__ V item_shift(const ItemDesc& it);
template <> __device__ __forceinline__ float2 item_shift<float2>(const ItemDesc& it) { return it.shiftf; }
template <> __device__ __forceinline__ double2 item_shift<double2>(const ItemDesc& it) { return it.shift; }
template <typename T> __device__ __forceinline__ const T* prob_diag(const ProblemDesc& pr);
template <> __device__ __forceinline__ const float* prob_diag<float>(const ProblemDesc& pr) { return pr.diagf; }
template <> __device__ __forceinline__ const double* prob_diag<double>(const ProblemDesc& pr) { return pr.diag; }
template <typename T> __device__ __forceinline__ T prob_a(const ProblemDesc& pr, int d);
template <> __device__ __forceinline__ float prob_a<float>(const ProblemDesc& pr, int d) { return pr.af[d]; }
template <> __device__ __forceinline__ double prob_a<double>(const ProblemDesc& pr, int d) { return pr.a[d]; }

// ---- grid barrier ---------------------------------------------------------

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// ---- bulk copies into shared memory (1D, completion on an mbarrier) ---------

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned long long* b, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
// One arrival that also announces the bytes the phase's copies will deliver.
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* b, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_test(unsigned long long* b, unsigned parity) {
    unsigned done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(smem_u32(b)), "r"(parity)
        : "memory");
    return done != 0;
}
// Global to shared copy of `bytes` (a multiple of 16; both addresses 16-byte
// aligned) whose completion is counted on mbarrier b.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* b) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(b))
                 : "memory");
}
// Orders this thread's generic-proxy accesses before its later bulk copies.
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async;" ::: "memory"); }

// Bounded wait for phase `parity` of mbarrier b.  On expiry the sticky error
// word is set and a second wait (at least 10 ms, whatever the limit) gives
// copies still in flight time to land before the buffer is reused or the CTA
// leaves; the launch then ends at its next barrier.
__device__ bool mbar_wait(unsigned long long* b, unsigned parity, int* err, unsigned long long timeout_ns) {
    unsigned long long t0 = global_ns();
    while (!mbar_test(b, parity)) {
        if (global_ns() - t0 > timeout_ns) {
            atomicExch(err, kErrTimeout);
            const unsigned long long drain = timeout_ns > 10000000ull ? timeout_ns : 10000000ull;
            t0 = global_ns();
            while (!mbar_test(b, parity) && global_ns() - t0 <= drain) {
            }
            return false;
        }
    }
    return true;
}

// All CTAs of the co-resident (cooperative) grid meet here.  bar[0] counts
// arrivals and is zeroed before every launch (the count never resets, so the
// barrier a CTA is at follows from the count its arrival returns).  Each CTA
// publishes its earlier writes with a fence and arrives with an atomic add,
// then waits with acquire loads until the count reaches the end of its
// barrier: the arrivals form a release sequence, so reading the final count
// synchronises with all of them and no CTA has to publish for the others.
// Every wait is bounded by timeout_ns; on expiry the sticky error word is set,
// a wait also ends when another CTA has set it, and every CTA leaves the
// kernel at its next barrier.  Returns false when the launch must end.
__device__ bool grid_sync(unsigned* bar, int* err, unsigned long long timeout_ns) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();                                   // the CTA's writes before its arrival
        const unsigned prev = atomicAdd(bar, 1u);
        const unsigned target = (prev / gridDim.x + 1u) * gridDim.x;   // arrivals that end this barrier
        const unsigned long long t0 = global_ns();
        while ((int)(ld_acquire_u32(bar) - target) < 0) {
            if (*(volatile int*)err != 0) break;
            if (global_ns() - t0 > timeout_ns) {
                atomicExch(err, kErrTimeout);
                break;
            }
        }
    }
    __syncthreads();
    return *(volatile int*)err == 0;
}

// Barrier that also timestamps the end of phase `code` (CTA 0 only).
// With the CTA trace on, every CTA also records when all its threads arrived.
__device__ __forceinline__ bool phase_sync(const EngineArgs& A, int code, int* tcount) {
    if (A.cta_trace != nullptr) {
        __syncthreads();
        const int c = *tcount;
        if (threadIdx.x == 0 && c < A.cta_trace_phases && (int)blockIdx.x < A.cta_trace_stride) {
            A.cta_trace[1 + (size_t)c * A.cta_trace_stride + blockIdx.x] = global_ns();
            if (blockIdx.x == 0) A.cta_trace[0] = (unsigned long long)(c + 1);
        }
    }
    const bool ok = grid_sync(A.bar, A.err, A.timeout_ns);
    if (threadIdx.x == 0) {
        const int c = *tcount;
        if (A.trace != nullptr && blockIdx.x == 0 && c < A.trace_cap) {
            A.trace[1 + 2 * c] = (unsigned long long)code;
            A.trace[2 + 2 * c] = global_ns();
            A.trace[0] = (unsigned long long)(c + 1);
        }
        *tcount = c + 1;
    }
    return ok;
}

// ---- reductions -------------------------------------------------------------

// Transpose-reduce NV per-lane values across a warp: afterwards lane l holds
// the warp-wide sum of value (l % NV); 31 shuffles for NV = 32.
template <int NV, typename T>
__device__ __forceinline__ T warp_transpose_reduce(T (&v)[NV], int lane) {
#pragma unroll
    for (int off = 16; off >= NV; off >>= 1) {
#pragma unroll
        for (int k = 0; k < NV; ++k) v[k] += __shfl_xor_sync(0xffffffffu, v[k], off);
    }
#pragma unroll
    for (int half = NV / 2; half >= 1; half >>= 1) {
        const bool up = (lane & half) != 0;
#pragma unroll
        for (int k = 0; k < half; ++k) {
            T send = up ? v[k] : v[k + half];
            T keep = up ? v[k + half] : v[k];
            v[k] = keep + __shfl_xor_sync(0xffffffffu, send, half);
        }
    }
    return v[0];
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

__device__ __forceinline__ double2 shfl2(double2 v, int src) {
    return make_double2(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
}

struct Smem {
    EngineArgs A;
    IOArgs io;
    unsigned long long mbar;       // completion of the X phase's bulk copies
    unsigned mphase;               // its current phase parity
    double2 red[kWarps][32];
    double redn[kWarps];
    double2 h1[kMaxM + 1];
    double2 h2[kMaxM + 1];
    double2 coef[kMaxM + 1];       // FP64 coefficients of the current item
    float2 coeff[kMaxM + 1];       // the same, rounded for the FP32 path
    double ssm[kMaxM + 1];
    double2 gsm[kMaxM + 1];
    double2 hfin[kMaxM + 2];       // Y: column j-1 completed
    double2 hnew[kMaxM + 2];       // Y: column j (pending)
    double2 coefG[kMaxM + 1];      // Y: coefficients of v_{j+1}
    float2 coefGf[kMaxM + 1];
    double yscal[4];               // Y: nu, s_j = t_j / nu, t_{j+1} = 1 / nu, 1 / t_j
    double gcs_s[kMaxM];           // Y: staged Givens cosines of the committed item
    double2 gsn_s[kMaxM];          //    and sines
    double2 ygq;                   // Y: gamma_j (coefficient of q_j in v_{j+1})
    int cnt[kBlock];
    int tls[kBlock];
    const double2* xptr[2 * kMaxPoles];
    double2 alpha[kMaxPoles];
    int nl;
    int ntasks;
    int kk;                        // Arnoldi steps of the current item (E2)
    bool xassign;                  // E2 writes x instead of adding (first update after a shared cycle)
    unsigned ep_now, ep_seen;      // Arnoldi-list epoch (delayed CGS2 loop)
    const void* basis;             // basis the current item's E2 reads
    double2* scratch;              // dynamic shared memory aliased with the staging tiles:
                                   // R (E2) or Hessenberg columns (Y), kScratch entries
    double2 yhat[kMaxM];           // PS: sum of alpha_k y_k of the poles completed on the shared basis
    int kyhat;                     //     its length (0: none)
    int nxlive;                    //     poles whose x the pole sum reads
    unsigned long long nbytes;     // algorithmic bytes this CTA moved (thread 0)
    unsigned long long nflops;     // FP64 flops of its arithmetic (thread 0)
    const void* gbasis;            //     the shared basis
};

template <typename V> __device__ __forceinline__ V coefg_at(const Smem& sm, int q);
template <> __device__ __forceinline__ float2 coefg_at<float2>(const Smem& sm, int q) { return sm.coefGf[q]; }
template <> __device__ __forceinline__ double2 coefg_at<double2>(const Smem& sm, int q) { return sm.coefG[q]; }
template <typename V> __device__ __forceinline__ V coef_at(const Smem& sm, int q);
template <> __device__ __forceinline__ float2 coef_at<float2>(const Smem& sm, int q) { return sm.coeff[q]; }
template <> __device__ __forceinline__ double2 coef_at<double2>(const Smem& sm, int q) { return sm.coef[q]; }

// CTA sum of NV complex values per thread; thread t < nvalid receives value t.
template <int NV, typename T>
__device__ __forceinline__ double2 cta_reduce_vec(Smem& sm, T (&re)[NV], T (&im)[NV], int nvalid) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T r = warp_transpose_reduce<NV, T>(re, lane);
    T i = warp_transpose_reduce<NV, T>(im, lane);
    if (lane < NV) sm.red[warp][lane] = make_double2((double)r, (double)i);
    __syncthreads();
    double2 out = make_double2(0.0, 0.0);
    if (threadIdx.x < nvalid) {
#pragma unroll
        for (int w = 0; w < kWarps; ++w) out = cadd(out, sm.red[w][threadIdx.x]);
    }
    __syncthreads();
    return out;
}

__device__ __forceinline__ double cta_reduce_scalar(Smem& sm, double v) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    v = warp_sum(v);
    if (lane == 0) sm.redn[warp] = v;
    __syncthreads();
    double out = 0.0;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int w = 0; w < kWarps; ++w) out += sm.redn[w];
    }
    __syncthreads();
    return out;   // valid in thread 0
}

// ---- work lists -------------------------------------------------------------

// List (in shared memory) of the items whose status bit is set in `mask`, and
// the prefix sums of their tile counts.  Identical in every CTA: statuses are
// read after a grid barrier and only changed in per-item phases.
// Tasks an item of the list gets: its tiles, or none for a pole starting its
// shared first cycle in a step launch when `e3` is set (its residual is b; the
// group item does the work and E4 reads the norm there).
__device__ __forceinline__ int list_tiles(const EngineArgs& A, int i, int s, bool e3) {
    const ItemDesc& it = A.item[i];
    if (e3 && s == ST_NEED_RES && A.mode == MODE_STEP && it.group >= 0 && ldi(&it.st->cycles) == 0) return 0;
    return it.ntiles;
}

__device__ void build_list(Smem& sm, int* list, int* prefix, unsigned mask, bool e3 = false) {
    const EngineArgs& A = sm.A;
    const int nit = A.nitems;
    const int per = (nit + kBlock - 1) / kBlock;
    const int i0 = threadIdx.x * per;
    const int i1 = min(nit, i0 + per);
    int c = 0, t = 0;
    for (int i = i0; i < i1; ++i) {
        const int s = ldi(&A.item[i].st->status);
        if (mask & (1u << s)) { ++c; t += list_tiles(A, i, s, e3); }
    }
    sm.cnt[threadIdx.x] = c;
    sm.tls[threadIdx.x] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ac = 0, at = 0;
        for (int k = 0; k < kBlock; ++k) {
            const int cc = sm.cnt[k], tt = sm.tls[k];
            sm.cnt[k] = ac;
            sm.tls[k] = at;
            ac += cc;
            at += tt;
        }
        sm.nl = ac;
        sm.ntasks = at;
        prefix[ac] = at;
    }
    __syncthreads();
    c = sm.cnt[threadIdx.x];
    t = sm.tls[threadIdx.x];
    for (int i = i0; i < i1; ++i) {
        const int s = ldi(&A.item[i].st->status);
        if (mask & (1u << s)) {
            list[c] = i;
            prefix[c] = t;
            ++c;
            t += list_tiles(A, i, s, e3);
        }
    }
    __syncthreads();
}

// Problems live in (backward) substep `sub`, with their tile prefix sums.
// The pole sum and the adjoint accumulation are FP64 work with no reuse:
// small tasks spread them over every SM.
constexpr int kPsPPT = 4;
constexpr int kPsTile = kBlock * kPsPPT;

__device__ void build_problem_list(Smem& sm, int* list, int* prefix, int sub) {
    const EngineArgs& A = sm.A;
    if (threadIdx.x == 0) {
        int c = 0, t = 0;
        for (int p = 0; p < A.nproblems; ++p) {
            if (sub < A.prob[p].nsub) {
                list[c] = p;
                prefix[c] = t;
                ++c;
                t += (A.prob[p].n + kPsTile - 1) / kPsTile;
            }
        }
        prefix[c] = t;
        sm.nl = c;
        sm.ntasks = t;
    }
    __syncthreads();
}

__device__ __forceinline__ int find_slot(const int* prefix, int nl, int task) {
    int lo = 0, hi = nl - 1;                  // largest l with prefix[l] <= task
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (prefix[mid] <= task) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// ---- stencil ----------------------------------------------------------------

struct Nb { int xm, xp, ym, yp, zm, zp; };

__device__ __forceinline__ Nb neighbours(int p, int nx, int ny, int nz) {
    Nb b;
    const int ix = p % nx;
    const int q = p / nx;
    const int iy = q % ny;
    const int iz = q / ny;
    b.xm = ix == 0 ? p + nx - 1 : p - 1;
    b.xp = ix == nx - 1 ? p - nx + 1 : p + 1;
    const int sy = nx;
    b.ym = iy == 0 ? p + sy * (ny - 1) : p - sy;
    b.yp = iy == ny - 1 ? p - sy * (ny - 1) : p + sy;
    const int sz = nx * ny;
    b.zm = iz == 0 ? p + sz * (nz - 1) : p - sz;
    b.zp = iz == nz - 1 ? p - sz * (nz - 1) : p + sz;
    return b;
}

// (A u)_p = sum_d a_d (u_{p+e_d} + u_{p-e_d}) + (diag_p - shift) u_p in precision
// T: the periodic second-order Laplacian of tau H with the diagonal tau (V - c)
// and the pole shift fused.
// t A u at point p with the scale t folded into the coefficients (at = t a_d,
// st = t shift): sum_d at_d (u_{p+e_d} + u_{p-e_d}) + (t diag_p - st) u_p.
// The arithmetic of t A u at one point from its loaded neighbours (x, y, z
// pairs; dims of them used) and diagonal entry dg.
template <typename T, typename V>
__device__ __forceinline__ V stencil_combine(V c, V xl, V xr, V yl, V yr, V zl, V zr, int dims, T dg, T t,
                                             T a0t, T a1t, T a2t, V st) {
    V s = mk2(a0t * (xl.x + xr.x), a0t * (xl.y + xr.y));
    if (dims > 1) {
        s.x += a1t * (yl.x + yr.x);
        s.y += a1t * (yl.y + yr.y);
    }
    if (dims > 2) {
        s.x += a2t * (zl.x + zr.x);
        s.y += a2t * (zl.y + zr.y);
    }
    // t = 1 and no shift (the shared basis after its first step): dd = dg
    // exactly, so the FMA is skipped (uniform branch)
    const T dd = (t == T(1) && st.x == T(0)) ? dg : fmat(dg, t, -st.x);
    s.x = fmat(dd, c.x, s.x);
    s.y = fmat(dd, c.y, s.y);
    if (st.y != T(0)) {                 // uniform: a shared basis has no shift
        s.x = fmat(st.y, c.y, s.x);
        s.y = fmat(-st.y, c.x, s.y);
    }
    return s;
}

template <typename T, typename V>
__device__ __forceinline__ V stencil_scaled(const V* __restrict__ u, int p, const ProblemDesc& pr,
                                            const T* __restrict__ diag, T t, T a0t, T a1t, T a2t, V st, V c) {
    const Nb b = neighbours(p, pr.nx, pr.ny, pr.nz);
    const int dims = 1 + (pr.ny > 1) + (pr.nz > 1);
    const V z = mk2(T(0), T(0));
    const V xl = ldv(u + b.xm), xr = ldv(u + b.xp);
    const V yl = dims > 1 ? ldv(u + b.ym) : z, yr = dims > 1 ? ldv(u + b.yp) : z;
    const V zl = dims > 2 ? ldv(u + b.zm) : z, zr = dims > 2 ? ldv(u + b.zp) : z;
    return stencil_combine<T, V>(c, xl, xr, yl, yr, zl, zr, dims, __ldg(diag + p), t, a0t, a1t, a2t, st);
}

// kL1: vector loads that may be served by L1 (ldv) or L2-only loads (ldp).
template <bool kL1, typename V> __device__ __forceinline__ V ldsel(const V* p) { return kL1 ? ldv(p) : ldp(p); }

template <typename T, typename V, bool kL1 = true>
__device__ __forceinline__ V stencil_apply(const V* __restrict__ u, int p, const ProblemDesc& pr,
                                           const T* __restrict__ diag, const T a0, const T a1,
                                           const T a2, const V shift) {
    const Nb b = neighbours(p, pr.nx, pr.ny, pr.nz);
    const V c = ldsel<kL1>(u + p);
    V s;
    {
        const V l = ldsel<kL1>(u + b.xm), r = ldsel<kL1>(u + b.xp);
        s = mk2(a0 * (l.x + r.x), a0 * (l.y + r.y));
    }
    if (pr.ny > 1) {
        const V l = ldsel<kL1>(u + b.ym), r = ldsel<kL1>(u + b.yp);
        s.x += a1 * (l.x + r.x);
        s.y += a1 * (l.y + r.y);
    }
    if (pr.nz > 1) {
        const V l = ldsel<kL1>(u + b.zm), r = ldsel<kL1>(u + b.zp);
        s.x += a2 * (l.x + r.x);
        s.y += a2 * (l.y + r.y);
    }
    const T dd = __ldg(diag + p) - shift.x;
    s.x = fmat(dd, c.x, s.x);
    s.y = fmat(dd, c.y, s.y);
    if (shift.y != T(0)) {
        s.x = fmat(shift.y, c.y, s.x);
        s.y = fmat(-shift.y, c.x, s.y);
    }
    return s;
}

// ---- per-problem state buffers ---------------------------------------------

// Problem q's state buffers; io holds the caller's pointers of this call.
__device__ __forceinline__ const double2* step_in(const IOArgs& io, const ProblemDesc& pr, int q, int sub) {
    if (sub == 0) return io.in[q];
    return (sub & 1) ? pr.tmp0 : pr.tmp1;
}
__device__ __forceinline__ double2* step_out(const IOArgs& io, const ProblemDesc& pr, int q, int sub) {
    if (sub == pr.nsub - 1) return io.out[q];
    return (sub & 1) ? pr.tmp1 : pr.tmp0;
}
// Backward substep bs = 0 undoes the last forward substep.
__device__ __forceinline__ const double2* adj_in(const IOArgs& io, const ProblemDesc& pr, int q, int bs) {
    if (bs == 0) return io.gout[q];
    return (bs & 1) ? pr.tmp0 : pr.tmp1;
}
__device__ __forceinline__ double2* adj_out(const IOArgs& io, const ProblemDesc& pr, int q, int bs) {
    if (bs == pr.nsub - 1) return io.out[q];
    return (bs & 1) ? pr.tmp1 : pr.tmp0;
}
__device__ __forceinline__ const double2* fwd_state(const IOArgs& io, const ProblemDesc& pr, int q, int bs) {
    const int s = pr.nsub - 1 - bs;
    return s == 0 ? io.in[q] : pr.ckpt + (size_t)s * (size_t)pr.n;
}
__device__ __forceinline__ const double2* item_rhs(int mode, const IOArgs& io, const ItemDesc& it,
                                                  const ProblemDesc& pr, int sub) {
    const int q = it.problem;
    if (mode == MODE_BACKWARD) return it.adjoint ? adj_in(io, pr, q, sub) : fwd_state(io, pr, q, sub);
    if (mode == MODE_SOLVE) return io.in[q];
    return step_in(io, pr, q, sub);
}

// ---- phases -------------------------------------------------------------------

// Partials are written once per "run": a maximal range of consecutive tiles of
// one item inside one CTA's share of the task range, at the slot of the run's
// first tile.  The partition (T tasks split evenly over G CTAs) is the same in
// every CTA, so a consumer can enumerate the run starts of an item itself.
__device__ __forceinline__ int range_start(int c, int T, int G) {
    const unsigned long long prod = (unsigned long long)c * (unsigned)T;     // 32-bit division when it fits
    return prod < (1ull << 32) ? (int)((unsigned)prod / (unsigned)G) : (int)(prod / (unsigned)G);
}
__device__ __forceinline__ int task_owner(int task, int T, int G) {
    return (int)((((long long)task + 1) * G - 1) / T);
}

// Runs of list slot l: candidate r (0 <= r < count) is the run of CTA c0 + r,
// starting at tile(r), or -1 when that CTA's share is empty (fewer tasks than
// CTAs: several CTAs then have the same start and only the last one owns it).
struct Runs {
    int t0, c0, count, T, G;
    __device__ __forceinline__ int tile(int r) const {
        if (r == 0) return 0;
        const int c = c0 + r;
        const int st = range_start(c, T, G);
        return st < range_start(c + 1, T, G) ? st - t0 : -1;
    }
};
__device__ __forceinline__ Runs item_runs(const int* prefix, int l, int T) {
    Runs R;
    R.T = T;
    R.G = gridDim.x;
    R.t0 = prefix[l];
    const int t1 = prefix[l + 1];
    R.c0 = task_owner(R.t0, T, R.G);
    R.count = task_owner(t1 - 1, T, R.G) - R.c0 + 1;
    return R;
}

// out[i] = scale_i * sum over the runs of item slot l of part[run][i], i < nv (nv <= 32).
// Each warp's lanes split into nvp-wide groups (nvp = nv rounded up to a power
// of two) that stride over the runs; the groups are summed with shuffles and
// the warps through shared memory (one block barrier).  AT is the accumulation
// type and the stored format: float2 partials where they are FP32 inner
// products (the one-reduction Arnoldi), double2 otherwise (CGS2).
template <typename AT>
__device__ void reduce_partials(Smem& sm, const double2* part, const ItemDesc& it, const Runs& R, int nv,
                                const double* scale, double2* out) {
    int nvp = 1;
    while (nvp < nv) nvp <<= 1;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int v = lane & (nvp - 1), rl = lane / nvp, rpw = 32 / nvp;
    AT ax = AT(0), ay = AT(0);
    if (v < nv) {
        const size_t off = (size_t)it.tile_off * sm.A.pv + v;
#pragma unroll 4
        for (int r = warp * rpw + rl; r < R.count; r += rpw * kWarps) {
            const int tl = R.tile(r);
            if (tl >= 0) {
                if (sizeof(AT) == 4) {
                    const float2 q = ldp((const float2*)part + off + (size_t)tl * sm.A.pv);
                    ax += (AT)q.x;
                    ay += (AT)q.y;
                } else {
                    const double2 q = ldp(part + off + (size_t)tl * sm.A.pv);
                    ax += (AT)q.x;
                    ay += (AT)q.y;
                }
            }
        }
    }
    for (int off = nvp; off < 32; off <<= 1) {
        ax += __shfl_xor_sync(0xffffffffu, ax, off);
        ay += __shfl_xor_sync(0xffffffffu, ay, off);
    }
    if (rl == 0) sm.red[warp][v] = make_double2((double)ax, (double)ay);
    __syncthreads();
    if (threadIdx.x < nv) {
        double2 s2 = make_double2(0.0, 0.0);
#pragma unroll
        for (int w = 0; w < kWarps; ++w) s2 = cadd(s2, sm.red[w][threadIdx.x]);
        out[threadIdx.x] = cscale(s2, scale[threadIdx.x]);
    }
    __syncthreads();
}

// Two partial sets at once (nv <= 16): one read loop, one block barrier.
__device__ void reduce_partials2(Smem& sm, const double2* partA, const double2* partB, const ItemDesc& it,
                                 const Runs& R, int nv, const double* scale, double2* outA, double2* outB) {
    int nvp = 1;
    while (nvp < nv) nvp <<= 1;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int v = lane & (nvp - 1), rl = lane / nvp, rpw = 32 / nvp;
    float ax = 0.f, ay = 0.f, bx = 0.f, by = 0.f;
    if (v < nv) {
        const size_t off = (size_t)it.tile_off * sm.A.pv + v;
#pragma unroll 4
        for (int r = warp * rpw + rl; r < R.count; r += rpw * kWarps) {
            const int tl = R.tile(r);
            if (tl >= 0) {
                const float2 qa = ldp((const float2*)partA + off + (size_t)tl * sm.A.pv);
                const float2 qb = ldp((const float2*)partB + off + (size_t)tl * sm.A.pv);
                ax += qa.x;
                ay += qa.y;
                bx += qb.x;
                by += qb.y;
            }
        }
    }
    for (int o = nvp; o < 32; o <<= 1) {
        ax += __shfl_xor_sync(0xffffffffu, ax, o);
        ay += __shfl_xor_sync(0xffffffffu, ay, o);
        bx += __shfl_xor_sync(0xffffffffu, bx, o);
        by += __shfl_xor_sync(0xffffffffu, by, o);
    }
    float2* redf = (float2*)sm.red;                                   // [kWarps][32]
    if (rl == 0) {
        redf[warp * 32 + v] = make_float2(ax, ay);
        redf[warp * 32 + 16 + v] = make_float2(bx, by);
    }
    __syncthreads();
    if (threadIdx.x < 2 * nv) {
        const int t = threadIdx.x < nv ? threadIdx.x : threadIdx.x - nv;
        const int col = threadIdx.x < nv ? t : 16 + t;
        float sx = 0.f, sy = 0.f;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) {
            const float2 q = redf[w * 32 + col];
            sx += q.x;
            sy += q.y;
        }
        (threadIdx.x < nv ? outA : outB)[t] = cscale(make_double2((double)sx, (double)sy), scale[t]);
    }
    __syncthreads();
}

// Warp-level sum of the norm partials of item slot l (all lanes get the sum).
__device__ __forceinline__ double warp_norm_partials(const ItemDesc& it, const Runs& R) {
    const int lane = threadIdx.x & 31;
    double ss = 0.0;
    for (int r = lane; r < R.count; r += 32) {
        const int tl = R.tile(r);
        if (tl >= 0) ss += ldd(it.partn + it.tile_off + tl);
    }
    return warp_sum(ss);
}

// First basis vector step j of the delayed CGS2 orthogonalises against.
__device__ __forceinline__ int win_start(const EngineArgs& A, int j) {
    return A.window > 0 ? max(0, j - A.window) : 0;
}

// Square of the residual estimate |g_{k+1}| of a cycle with k columns taken
// as a bound on the true residual: with a windowed basis the columns are
// orthonormal only locally, and ||r|| <= sqrt(k + 1) |g_{k+1}| (unit columns).
// Squared, so the per-step test needs no square root.
__device__ __forceinline__ double res2_bound(const EngineArgs& A, double2 g, int k) {
    const double r2 = g.x * g.x + g.y * g.y;
    return A.window > 0 ? r2 * (double)(k + 1) : r2;
}

// y = R^{-1} g for the packed upper triangle R (column l at l(l+1)/2) in
// shared memory, k <= 64, by one warp: lane i holds rows i and i + 32 and the
// columns are eliminated from the last; y lands in shared memory.
__device__ void back_substitute(const double2* R, const double2* g, double2* y, int k, int win) {
    const int lane = threadIdx.x & 31;
    double2 a0 = lane < k ? g[lane] : make_double2(0.0, 0.0);
    double2 a1 = lane + 32 < k ? g[lane + 32] : make_double2(0.0, 0.0);
    for (int l = k - 1; l >= 0; --l) {
        const double2* col = R + l * (l + 1) / 2;
        double2 yl = make_double2(0.0, 0.0);
        if (lane == (l & 31)) {
            const double2 d = col[l];
            const double2 a = l < 32 ? a0 : a1;
            const double den = d.x * d.x + d.y * d.y;
            if (den > 0.0) yl = cscale(cmul(a, cconj(d)), 1.0 / den);
            y[l] = yl;
        }
        yl = shfl2(yl, l & 31);
        const int lo = win > 0 ? max(0, l - win - 1) : 0;   // a windowed column is zero above row lo
        if (lane < l && lane >= lo) a0 = csub(a0, cmul(col[lane], yl));
        if (lane + 32 < l && lane + 32 >= lo) a1 = csub(a1, cmul(col[lane + 32], yl));
    }
    __syncwarp();
}

// Algorithmic byte count: points of a run times the bytes a point moves.
__device__ __forceinline__ long long run_points(int n, int tile, int tb, int te) {
    return (long long)min(n, te * tile) - (long long)tb * tile;
}
__device__ __forceinline__ void acct(Smem& sm, long long pts, long long bytes_per_point) {
    if (threadIdx.x == 0) sm.nbytes += (unsigned long long)(pts * bytes_per_point);
}
// FP64 flop count (an FMA is two): only the arithmetic done in double.
__device__ __forceinline__ void acctf(Smem& sm, long long pts, long long flops_per_point) {
    if (threadIdx.x == 0) sm.nflops += (unsigned long long)(pts * flops_per_point);
}
// Flops of one application of the (2d+1)-point complex stencil with the shift.
__device__ __forceinline__ long long stencil_flops(const ProblemDesc& pr) {
    const int d = 1 + (pr.ny > 1) + (pr.nz > 1);
    return 6 * d + 8;
}

__device__ __forceinline__ void load_scales(Smem& sm, const ItemState* S, int cnt) {
    if (threadIdx.x < cnt) sm.ssm[threadIdx.x] = ldd(&S->s[threadIdx.x]);
    __syncthreads();
}

template <typename T, int VG, int MINB>
struct Phases {
    typedef typename C2<T>::t V;
    // points per thread held at once in the update sweeps: FP64 accumulators
    // of 8 points fit the register budget of one CTA per SM, not of two
    static constexpr int kChunk = (sizeof(T) == 8 && MINB > 1) ? kPPT / 2 : kPPT;

    // Every thread owns points p0 + r * kBlock + threadIdx.x, r < kPPT, of a
    // tile; per basis vector all of its kPPT loads are independent.  A CTA
    // walks the tiles [tb, te) of one item (a run) accumulating its partial
    // sums in registers and reduces them once per run.

    // E3: residual r = b - A x (FP64), stored as u_0; x = 0 on the first cycle.
    static __device__ void e3(Smem& sm, int sub, int item, int tb, int te) {
        const EngineArgs& A = sm.A;
        const ItemDesc& it = A.item[item];
        const int it_n = it.n, it_tile = it.tile;
        const ProblemDesc& pr = A.prob[it.problem];
        const int cycles = ldi(&it.st->cycles);
        // a pole starting its shared first cycle in a step launch: its residual is b,
        // whose norm the group item computes (E4 reads it there)
        if (cycles == 0 && A.mode == MODE_STEP && it.group >= 0) return;
        const double2* b = item_rhs(A.mode, sm.io, it, pr, sub);
        V* U = (V*)it.basis;
        double2* x = it.x;
        double acc = 0.0;
        acct(sm, run_points(it_n, it_tile, tb, te),
             16 + (cycles > 0 ? 16 + 8 : (x != nullptr && !(A.mode == MODE_STEP && it.group >= 0) ? 16 : 0)) +
                 ((it.group >= 0 && cycles == 0) ? 0 : (long long)sizeof(V)));
        acctf(sm, run_points(it_n, it_tile, tb, te), cycles > 0 ? stencil_flops(pr) + 6 : 4);
        for (int tile = tb; tile < te; ++tile) {
            const int p0 = tile * it_tile, pend = min(it_n, p0 + it_tile);
            double2 rv[kPPT];
#pragma unroll
            for (int r = 0; r < kPPT; ++r) {
                const int p = p0 + r * kBlock + threadIdx.x;
                rv[r] = p < pend ? ldv(b + p) : make_double2(0.0, 0.0);
            }
            if (cycles == 0) {
                // x0 = 0; in a step launch a pole on a shared first cycle gets x assigned by its
                // first update, or never reads it (finished on the shared basis, or b = 0)
                if (x != nullptr && !(A.mode == MODE_STEP && it.group >= 0)) {
#pragma unroll
                    for (int r = 0; r < kPPT; ++r) {
                        const int p = p0 + r * kBlock + threadIdx.x;
                        if (p < pend) x[p] = make_double2(0.0, 0.0);
                    }
                }
            } else {
#pragma unroll
                for (int r = 0; r < kPPT; ++r) {
                    const int p = p0 + r * kBlock + threadIdx.x;
                    if (p < pend)
                        rv[r] = csub(rv[r], stencil_apply<double, double2>(x, p, pr, pr.diag, pr.a[0], pr.a[1],
                                                                            pr.a[2], it.shift));
                }
            }
            // a pole whose first cycle runs on its group's basis needs no u_0
            const bool store = !(it.group >= 0 && cycles == 0);
#pragma unroll
            for (int r = 0; r < kPPT; ++r) {
                const int p = p0 + r * kBlock + threadIdx.x;
                if (p < pend) {
                    if (store) U[p] = cvt2<V>(rv[r]);
                    acc += rv[r].x * rv[r].x + rv[r].y * rv[r].y;
                }
            }
        }
        const double tot = cta_reduce_scalar(sm, acc);
        if (threadIdx.x == 0) it.partn[it.tile_off + tb] = tot;
    }

    // Dot sweeps: the tile of w sits in shared memory (ws); each warp owns up
    // to 4 basis vectors (or, when there are fewer vectors than warps, a row
    // range of one vector), so the per-lane accumulators stay in a few
    // registers and a run needs one reduction.
    struct DotPlan {
        int nvec;
        int q[4];
        int row0, row1;        // rows of 32 points of the tile
    };
    static __device__ __forceinline__ DotPlan dot_plan(int J, int tile) {
        const int wp = threadIdx.x >> 5;
        const int rows = tile / 32;
        DotPlan d;
        d.nvec = 0;
        if (J >= kWarps) {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int q = wp + kWarps * k;
                d.q[k] = q;
                if (q < J) d.nvec = k + 1;
            }
            d.row0 = 0;
            d.row1 = rows;
        } else {
            const int vpw = kWarps / J;
            const int q = wp / vpw;
            d.q[0] = d.q[1] = d.q[2] = d.q[3] = q;
            if (q < J) {
                d.nvec = 1;
                const int ch = wp - q * vpw;
                d.row0 = ch * rows / vpw;
                d.row1 = (ch + 1) * rows / vpw;
            } else {
                d.row0 = d.row1 = 0;
            }
        }
        return d;
    }

    // acc[s] += sum over the warp's rows of conj(u_q) w for the warp's vectors.
    static __device__ __forceinline__ void dot_tile(const V* U, size_t n, const V* ws, int p0, int pend,
                                                    const DotPlan& d, T (&ar)[4], T (&ai)[4]) {
        const int lane = threadIdx.x & 31;
        for (int sl = 0; sl < d.nvec; ++sl) {
            const V* uq = U + (size_t)d.q[sl] * n + p0;
            T sr = T(0), si = T(0);
            for (int row = d.row0; row < d.row1; row += 8) {
                V u[8];
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const int pl = (row + k) * 32 + lane;
                    u[k] = (row + k < d.row1 && p0 + pl < pend) ? ldv(uq + pl) : mk2(T(0), T(0));
                }
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    if (row + k < d.row1) {
                        const V w = ws[(row + k) * 32 + lane];
                        sr += u[k].x * w.x + u[k].y * w.y;
                        si += u[k].x * w.y - u[k].y * w.x;
                    }
                }
            }
            // slot sl of this warp (fixed unrolled index to stay in registers)
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                if (k == sl) { ar[k] += sr; ai[k] += si; }
            }
        }
    }

    // End of a run: partial dots of the warps' vectors into part[tb][0..J),
    // stored as float2 (kF32: the one-reduction Arnoldi) or double2 (CGS2).
    template <bool kF32, typename AT>
    static __device__ void dot_finish(Smem& sm, const ItemDesc& it, double2* part, int tb, int J,
                                      const DotPlan& d, AT (&ar)[4], AT (&ai)[4]) {
        const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const AT r = warp_sum(ar[k]);
            const AT i = warp_sum(ai[k]);
            if (lane == 0) sm.red[wp][k] = make_double2((double)r, (double)i);
        }
        __syncthreads();
        if (threadIdx.x < J) {
            const int q = threadIdx.x;
            double2 acc = make_double2(0.0, 0.0);
            if (J >= kWarps) {
                acc = sm.red[q % kWarps][q / kWarps];
            } else {
                const int vpw = kWarps / J;
                for (int w = q * vpw; w < (q + 1) * vpw; ++w) acc = cadd(acc, sm.red[w][0]);
            }
            const size_t at = (size_t)(it.tile_off + tb) * sm.A.pv + q;
            if (kF32) ((float2*)part)[at] = make_float2((float)acc.x, (float)acc.y);
            else part[at] = acc;
        }
        __syncthreads();
    }

    // Both partial sets of the one-reduction Arnoldi in one pass (one barrier
    // fewer): warps' sums of (ar, ai) in red[w][0..4), of (br, bi) in red[w][4..8).
    static __device__ void dot_finish2(Smem& sm, const ItemDesc& it, int tb, int J, const DotPlan& d,
                                       float (&ar)[4], float (&ai)[4], float (&br)[4], float (&bi)[4]) {
        const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float r = warp_sum(ar[k]), i = warp_sum(ai[k]);
            const float r2 = warp_sum(br[k]), i2 = warp_sum(bi[k]);
            if (lane == 0) {
                sm.red[wp][k] = make_double2((double)r, (double)i);
                sm.red[wp][4 + k] = make_double2((double)r2, (double)i2);
            }
        }
        __syncthreads();
        const int q = threadIdx.x & 31, set = threadIdx.x >> 5;      // warp 0: first set, warp 1: second
        if (set < 2 && q < J) {
            double2 acc = make_double2(0.0, 0.0);
            if (J >= kWarps) {
                acc = sm.red[q % kWarps][4 * set + q / kWarps];
            } else {
                const int vpw = kWarps / J;
                for (int w = q * vpw; w < (q + 1) * vpw; ++w) acc = cadd(acc, sm.red[w][4 * set]);
            }
            ((float2*)(set == 0 ? it.part1 : it.part2))[(size_t)(it.tile_off + tb) * sm.A.pv + q] =
                make_float2((float)acc.x, (float)acc.y);
        }
        __syncthreads();
    }

    // w[r] -= sum_{q <= j} c_q u_q at the thread's points.
    static __device__ __forceinline__ void subtract(const Smem& sm, const V* U, size_t n, V (&w)[kPPT], int p0,
                                                    int pend, int j) {
#pragma unroll 2
        for (int q = 0; q <= j; ++q) {
            const V* uq = U + (size_t)q * n;
            const V c = coef_at<V>(sm, q);
#pragma unroll
            for (int r = 0; r < kPPT; ++r) {
                const int p = p0 + r * kBlock + threadIdx.x;
                const V u = p < pend ? ldv(uq + p) : mk2(T(0), T(0));
                w[r] = cfms(w[r], c, u);
            }
        }
    }

    static __device__ __forceinline__ void load_tile(const V* src, V (&w)[kPPT], int p0, int pend) {
#pragma unroll
        for (int r = 0; r < kPPT; ++r) {
            const int p = p0 + r * kBlock + threadIdx.x;
            w[r] = p < pend ? ldv(src + p) : mk2(T(0), T(0));
        }
    }

    static __device__ __forceinline__ void stage_tile(V* ws, const V (&w)[kPPT]) {
#pragma unroll
        for (int r = 0; r < kPPT; ++r) ws[r * kBlock + threadIdx.x] = w[r];
    }

    // P1: w = A (s_j u_j) into slot j+1; p1_i = sum conj(u_i) w, i <= j.
    static __device__ void p1(Smem& sm, V* ws, int item, int tb, int te, int j) {
        const EngineArgs& A = sm.A;
        const ItemDesc& it = A.item[item];
        const int it_n = it.n, it_tile = it.tile;
        acct(sm, run_points(it_n, it_tile, tb, te), (j + 3) * (long long)sizeof(V) + (long long)sizeof(T));
        const ProblemDesc& pr = A.prob[it.problem];
        if (sizeof(T) == 8) acctf(sm, run_points(it_n, it_tile, tb, te), stencil_flops(pr) + 2 + 8 * (j + 1));
        const size_t n = (size_t)it_n;
        V* U = (V*)it.basis;
        const V* uj = U + (size_t)j * n;
        V* wv = U + (size_t)(j + 1) * n;
        const T sj = (T)ldd(&it.st->s[j]);
        const V shift = item_shift<V>(it);
        const T* diag = prob_diag<T>(pr);
        const T a0 = prob_a<T>(pr, 0), a1 = prob_a<T>(pr, 1), a2 = prob_a<T>(pr, 2);
        const DotPlan d = dot_plan(j + 1, it_tile);
        T ar[4] = {T(0), T(0), T(0), T(0)}, ai[4] = {T(0), T(0), T(0), T(0)};
        for (int tile = tb; tile < te; ++tile) {
            const int p0 = tile * it_tile, pend = min(it_n, p0 + it_tile);
            V w[kPPT];
#pragma unroll
            for (int r = 0; r < kPPT; ++r) {
                const int p = p0 + r * kBlock + threadIdx.x;
                if (p < pend) {
                    V v = stencil_apply<T, V>(uj, p, pr, diag, a0, a1, a2, shift);
                    v.x *= sj;
                    v.y *= sj;
                    w[r] = v;
                    wv[p] = v;
                } else {
                    w[r] = mk2(T(0), T(0));
                }
            }
            stage_tile(ws, w);
            __syncthreads();
            dot_tile(U, n, ws, p0, pend, d, ar, ai);
            __syncthreads();
        }
        dot_finish<false>(sm, it, it.part1, tb, j + 1, d, ar, ai);
    }

    // P2 prologue: h1_i = s_i sum p1_i; coefficients s_i h1_i of u_i.
    static __device__ void p2_pro(Smem& sm, int item, const Runs& R, int j) {
        const ItemDesc& it = sm.A.item[item];
        load_scales(sm, it.st, j + 1);
        reduce_partials<double>(sm, it.part1, it, R, j + 1, sm.ssm, sm.h1);
        if (threadIdx.x <= j) {
            const double2 c = cscale(sm.h1[threadIdx.x], sm.ssm[threadIdx.x]);
            sm.coef[threadIdx.x] = c;
            sm.coeff[threadIdx.x] = make_float2((float)c.x, (float)c.y);
        }
        __syncthreads();
    }

    // P2: w' = w - sum_i c_i u_i (staged in shared memory); p2_i = sum conj(u_i) w'.
    static __device__ void p2(Smem& sm, V* ws, int item, int tb, int te, int j) {
        const ItemDesc& it = sm.A.item[item];
        const int it_n = it.n, it_tile = it.tile;
        acct(sm, run_points(it_n, it_tile, tb, te), (2 * j + 3) * (long long)sizeof(V));
        if (sizeof(T) == 8) acctf(sm, run_points(it_n, it_tile, tb, te), 16 * (j + 1));
        const size_t n = (size_t)it_n;
        const V* U = (const V*)it.basis;
        const V* wv = U + (size_t)(j + 1) * n;
        const DotPlan d = dot_plan(j + 1, it_tile);
        T ar[4] = {T(0), T(0), T(0), T(0)}, ai[4] = {T(0), T(0), T(0), T(0)};
        for (int tile = tb; tile < te; ++tile) {
            const int p0 = tile * it_tile, pend = min(it_n, p0 + it_tile);
            V w[kPPT];
            load_tile(wv, w, p0, pend);
            subtract(sm, U, n, w, p0, pend, j);
            stage_tile(ws, w);
            __syncthreads();
            dot_tile(U, n, ws, p0, pend, d, ar, ai);
            __syncthreads();
        }
        dot_finish<false>(sm, it, it.part2, tb, j + 1, d, ar, ai);
    }

    // P3 prologue: h = h1 + h2; coefficients s_i h_i.
    static __device__ void p3_pro(Smem& sm, int item, const Runs& R, int j) {
        const ItemDesc& it = sm.A.item[item];
        load_scales(sm, it.st, j + 1);
        reduce_partials<double>(sm, it.part1, it, R, j + 1, sm.ssm, sm.h1);
        reduce_partials<double>(sm, it.part2, it, R, j + 1, sm.ssm, sm.h2);
        if (threadIdx.x <= j) {
            const double2 h = cadd(sm.h1[threadIdx.x], sm.h2[threadIdx.x]);
            sm.h1[threadIdx.x] = h;
            const double2 c = cscale(h, sm.ssm[threadIdx.x]);
            sm.coef[threadIdx.x] = c;
            sm.coeff[threadIdx.x] = make_float2((float)c.x, (float)c.y);
        }
        __syncthreads();
    }

    // P3: w <- w - sum_i c_i u_i (stored), ||w||^2; the run starting at tile 0
    // publishes the Hessenberg column.
    static __device__ void p3(Smem& sm, int item, int tb, int te, int j) {
        const ItemDesc& it = sm.A.item[item];
        const int it_n = it.n, it_tile = it.tile;
        acct(sm, run_points(it_n, it_tile, tb, te), (j + 3) * (long long)sizeof(V));
        if (sizeof(T) == 8) acctf(sm, run_points(it_n, it_tile, tb, te), 8 * (j + 1) + 4);
        const size_t n = (size_t)it_n;
        V* U = (V*)it.basis;
        V* wv = U + (size_t)(j + 1) * n;
        if (tb == 0 && threadIdx.x <= j) it.st->hcol[threadIdx.x] = sm.h1[threadIdx.x];
        T acc = T(0);
        for (int tile = tb; tile < te; ++tile) {
            const int p0 = tile * it_tile, pend = min(it_n, p0 + it_tile);
            V w[kPPT];
            load_tile(wv, w, p0, pend);
            subtract(sm, U, n, w, p0, pend, j);
#pragma unroll
            for (int r = 0; r < kPPT; ++r) {
                const int p = p0 + r * kBlock + threadIdx.x;
                if (p < pend) {
                    wv[p] = w[r];
                    acc += w[r].x * w[r].x + w[r].y * w[r].y;
                }
            }
        }
        const double tot = cta_reduce_scalar(sm, (double)acc);
        if (threadIdx.x == 0) it.partn[it.tile_off + tb] = tot;
    }

    // ---- delayed CGS2 (one global reduction per Arnoldi step) -------------
    //
    // Entering step j, slots 0..j-1 hold the (locally) orthonormal q_0..q_{j-1}
    // up to their scales (q_i = s_i u_i) and slot j holds v_j = t_j u_j: A q_{j-1}
    // projected once against them (j = 0: the residual, t_0 = 1/beta).  X
    // computes w = A v_j and, in the same sweep,
    // a = Q^H v_j, c = v_j^H v_j, b = Q^H w, d = v_j^H w.  Y reorthogonalises
    // and normalises v_j (q_j = (v_j - Q a)/nu, nu^2 = c - |a|^2), which
    // completes Hessenberg column j-1 (h += a, h_{j,j-1} = nu), and uses the
    // Arnoldi relation A Q = Q_j H to form column j of A q_j = (w - Q_j H a)/nu
    // and the next candidate v_{j+1} = A q_j - Q_j h_{:,j} in one sweep.

    // Two dot products per basis vector in one read: with the v tile and the w
    // tile, both staged in FP32.  The dot products only choose the
    // orthogonalisation coefficients; the update sweep applies them in the
    // basis precision, which keeps the Arnoldi relation A Q = Q H to that
    // precision whatever their accuracy (FP32 dots leave the columns
    // orthonormal to ~1e-7, well inside the residual bound's slack).
    static __device__ __forceinline__ void dot_tile2(const V* U, size_t n, const float2* wsv, const float2* wsw,
                                                     int p0, int pend, const DotPlan& d, bool withw, float (&ar)[4],
                                                     float (&ai)[4], float (&br)[4], float (&bi)[4]) {
        const int lane = threadIdx.x & 31;
        for (int sl = 0; sl < d.nvec; ++sl) {
            const V* uq = U + (size_t)d.q[sl] * n + p0;
            float sr = 0.f, si = 0.f, tr = 0.f, ti = 0.f;
            for (int row = d.row0; row < d.row1; row += 8) {
                float2 u[8];
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const int pl = (row + k) * 32 + lane;
                    u[k] = (row + k < d.row1 && p0 + pl < pend) ? dot_f2(ldv(uq + pl)) : make_float2(0.f, 0.f);
                }
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    if (row + k < d.row1) {
                        const int pl = (row + k) * 32 + lane;
                        const float2 v = wsv[pl];
                        sr += u[k].x * v.x + u[k].y * v.y;
                        si += u[k].x * v.y - u[k].y * v.x;
                        if (withw) {
                            const float2 w = wsw[pl];
                            tr += u[k].x * w.x + u[k].y * w.y;
                            ti += u[k].x * w.y - u[k].y * w.x;
                        }
                    }
                }
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                if (k == sl) { ar[k] += sr; ai[k] += si; br[k] += tr; bi[k] += ti; }
            }
        }
    }

    static __device__ void dx(Smem& sm, V* wsv, V* wsw, int item, int tb, int te, int j, bool matvec) {
        const EngineArgs& A = sm.A;
        const ItemDesc& it = A.item[item];
        const int it_n = it.n, it_tile = it.tile;
        const ProblemDesc& pr = A.prob[it.problem];
        const size_t n = (size_t)it_n;
        V* U = (V*)it.basis;
        const V* uj = U + (size_t)j * n;
        V* wv = U + (size_t)(j + 1) * n;
        // v_j = t_j x slot j (t_0 = 1/beta; later t_j = 1/nu_{j-1}, set by the
        // previous step's commit)
        const T tj = (T)ldp(&it.st->vt[j & 1]).x;
        const V shift = item_shift<V>(it);
        const T* diag = prob_diag<T>(pr);
        const T a0 = prob_a<T>(pr, 0), a1 = prob_a<T>(pr, 1), a2 = prob_a<T>(pr, 2);
        const int j0 = win_start(A, j);                     // dots with q_j0 .. q_{j-1} and v_j
        const V* U0 = U + (size_t)j0 * n;
        const T a0t = a0 * tj, a1t = a1 * tj, a2t = a2 * tj;   // t_j folded into the stencil
        const V sht = mk2(shift.x * tj, shift.y * tj);
        const float tjf = (float)tj;
        float2* fsv = (float2*)wsv;                         // FP32 copies of the v and w tiles
        float2* fsw = (float2*)wsw;
        acct(sm, run_points(it_n, it_tile, tb, te),
             (j - j0 + 1) * (long long)sizeof(V) + (matvec ? (long long)sizeof(V) + (long long)sizeof(T) : 0));
        if (sizeof(T) == 8)
            acctf(sm, run_points(it_n, it_tile, tb, te), matvec ? stencil_flops(pr) : 0);
        if (matvec && j + 1 - j0 <= 4) {
            // staged neighbours: FP64 basis (16-byte entries, so every piece is a
            // legal bulk copy), one CTA per SM (registers for the prefetched
            // vectors), 1D/2D grids whose tile and halos fit the buffer
            const int halo = pr.ny > 1 ? pr.nx : 1;
            if (sizeof(T) == 8 && MINB == 1 && pr.nz == 1 && it_tile + 2 * halo <= 2 * kTile)
                dx_window_staged(sm, wsv, it, U0, uj, wv, n, pr, diag, tj, a0t, a1t, a2t, sht, tjf, tb, te,
                                 j + 1 - j0);
            else
                dx_window(sm, it, U0, uj, wv, n, pr, diag, tj, a0t, a1t, a2t, sht, tjf, tb, te, j + 1 - j0);
            return;
        }
        const DotPlan d = dot_plan(j + 1 - j0, it_tile);
        float ar[4] = {0.f, 0.f, 0.f, 0.f}, ai[4] = {0.f, 0.f, 0.f, 0.f};   // FP32 inner products
        float br[4] = {0.f, 0.f, 0.f, 0.f}, bi[4] = {0.f, 0.f, 0.f, 0.f};
        for (int tile = tb; tile < te; ++tile) {
            const int p0 = tile * it_tile, pend = min(it_n, p0 + it_tile);
#pragma unroll
            for (int r = 0; r < kPPT; ++r) {
                const int p = p0 + r * kBlock + threadIdx.x;
                float2 vf = make_float2(0.f, 0.f);
                V w = mk2(T(0), T(0));
                if (p < pend) {
                    const V u = ldv(uj + p);
                    const float2 uf = dot_f2(u);
                    vf = make_float2(tjf * uf.x, tjf * uf.y);      // v_j = t_j u_j, only its FP32 copy is needed
                    if (matvec) {
                        w = stencil_scaled<T, V>(uj, p, pr, diag, tj, a0t, a1t, a2t, sht, u);
                        wv[p] = w;
                    }
                }
                fsv[r * kBlock + threadIdx.x] = vf;
                fsw[r * kBlock + threadIdx.x] = dot_f2(w);
            }
            __syncthreads();
            dot_tile2(U0, n, fsv, fsw, p0, pend, d, matvec, ar, ai, br, bi);
            __syncthreads();
        }
        if (matvec) dot_finish2(sm, it, tb, j + 1 - j0, d, ar, ai, br, bi);
        else dot_finish<true>(sm, it, it.part1, tb, j + 1 - j0, d, ar, ai);
    }

    // X for a step with at most 4 vectors in the window (slots j0 .. j): every
    // thread accumulates the FP32 inner products of its own points inside the
    // stencil sweep, so the window vectors' loads overlap the stencil's and
    // the tile needs no staging pass.  The run's partials are a warp
    // transpose-reduce and a fixed-order sum over the warps, in the layout of
    // the staged path (part1: a and c, part2: b and d).
    static __device__ void dx_window(Smem& sm, const ItemDesc& it, const V* U0, const V* uj, V* wv, size_t n,
                                     const ProblemDesc& pr, const T* diag, T tj, T a0t, T a1t, T a2t, V sht,
                                     float tjf, int tb, int te, int J) {
        const int it_n = it.n, it_tile = it.tile;
        float v[16];                      // [2k, 2k+1]: conj(u_k) v_j; [8 + 2k, 9 + 2k]: conj(u_k) w
#pragma unroll
        for (int k = 0; k < 16; ++k) v[k] = 0.f;
        for (int tile = tb; tile < te; ++tile) {
            const int p0 = tile * it_tile, pend = min(it_n, p0 + it_tile);
#pragma unroll
            for (int r = 0; r < kPPT; ++r) {
                const int p = p0 + r * kBlock + threadIdx.x;
                if (p < pend) {
                    const V u = ldv(uj + p);
                    const V w = stencil_scaled<T, V>(uj, p, pr, diag, tj, a0t, a1t, a2t, sht, u);
                    wv[p] = w;
                    const float2 uf = dot_f2(u), wf = dot_f2(w);
                    const float2 vf = make_float2(tjf * uf.x, tjf * uf.y);
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        if (k < J) {
                            const float2 q = k < J - 1 ? dot_f2(ldv(U0 + (size_t)k * n + p)) : uf;
                            v[2 * k] = fmaf(q.x, vf.x, fmaf(q.y, vf.y, v[2 * k]));
                            v[2 * k + 1] = fmaf(q.x, vf.y, fmaf(-q.y, vf.x, v[2 * k + 1]));
                            v[8 + 2 * k] = fmaf(q.x, wf.x, fmaf(q.y, wf.y, v[8 + 2 * k]));
                            v[9 + 2 * k] = fmaf(q.x, wf.y, fmaf(-q.y, wf.x, v[9 + 2 * k]));
                        }
                    }
                }
            }
        }
        window_finish(sm, it, tb, J, v);
    }

    // The run's partials of a windowed X step from the per-thread sums v.
    static __device__ void window_finish(Smem& sm, const ItemDesc& it, int tb, int J, float (&v)[16]) {
        const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
        const float sre = warp_transpose_reduce<16, float>(v, lane);       // lane l: value l % 16
        const float sim = __shfl_down_sync(0xffffffffu, sre, 1);
        float2* redf = (float2*)sm.red;                                   // [kWarps][8]
        if (lane < 16 && (lane & 1) == 0) redf[wp * 8 + (lane >> 1)] = make_float2(sre, sim);
        __syncthreads();
        const int q = threadIdx.x & 31, set = threadIdx.x >> 5;          // warp 0: a, c; warp 1: b, d
        if (set < 2 && q < J) {
            float2 acc = make_float2(0.f, 0.f);
            for (int w = 0; w < kWarps; ++w) {
                const float2 t = redf[w * 8 + 4 * set + q];
                acc.x += t.x;
                acc.y += t.y;
            }
            ((float2*)(set == 0 ? it.part1 : it.part2))[(size_t)(it.tile_off + tb) * sm.A.pv + q] = acc;
        }
        __syncthreads();
    }

    // dx_window on a 1D or 2D grid with the staging buffer `stage` (2 kTile
    // vector entries): the tile and one halo on each side (a row in 2D, a
    // point in 1D) form a contiguous range of points up to the periodic wrap,
    // which at most three bulk copies bring into shared memory; the window
    // vectors and the diagonal of the thread's points are loaded meanwhile,
    // and the stencil reads its neighbours from the staged range.  The
    // arithmetic is the one of dx_window (stencil_combine), point by point.
    static __device__ void dx_window_staged(Smem& sm, V* stage, const ItemDesc& it, const V* U0, const V* uj,
                                            V* wv, size_t n, const ProblemDesc& pr, const T* diag, T tj, T a0t,
                                            T a1t, T a2t, V sht, float tjf, int tb, int te, int J) {
        const int it_n = it.n, it_tile = it.tile;
        const int nx = pr.nx;
        const bool two = pr.ny > 1;
        const int H = two ? nx : 1;
        const V zero = mk2(T(0), T(0));
        unsigned par = sm.mphase;                   // written by thread 0 before the last grid barrier
        float v[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) v[k] = 0.f;
        for (int tile = tb; tile < te; ++tile) {
            const int p0 = tile * it_tile, pend = min(it_n, p0 + it_tile);
            const int cnt = pend - p0 + 2 * H;      // staged points p0 - H .. pend + H - 1 (mod n)
            __syncthreads();                        // earlier readers of the buffer are done
            if (threadIdx.x == 0) {
                fence_proxy_async();
                mbar_expect_tx(&sm.mbar, (unsigned)cnt * (unsigned)sizeof(V));
                for (int done = 0; done < cnt;) {
                    int g = p0 - H + done;
                    g = g < 0 ? g + it_n : (g >= it_n ? g - it_n : g);
                    const int len = min(cnt - done, it_n - g);
                    bulk_g2s(stage + done, uj + g, (unsigned)len * (unsigned)sizeof(V), &sm.mbar);
                    done += len;
                }
            }
            V q0[kPPT], q1[kPPT], q2[kPPT];
            T dg[kPPT];
#pragma unroll
            for (int r = 0; r < kPPT; ++r) {
                const int p = p0 + r * kBlock + threadIdx.x;
                const bool in = p < pend;
                dg[r] = in ? __ldg(diag + p) : T(0);
                q0[r] = (in && J > 1) ? ldv(U0 + p) : zero;
                q1[r] = (in && J > 2) ? ldv(U0 + n + p) : zero;
                q2[r] = (in && J > 3) ? ldv(U0 + 2 * n + p) : zero;
            }
            mbar_wait(&sm.mbar, par, sm.A.err, sm.A.timeout_ns);
            par ^= 1u;
            // x index of the thread's point: one division per tile, then steps
            // of kBlock mod nx (each at most one wrap)
            const int xstep = two ? kBlock % nx : 0;
            int ix = two ? (p0 + (int)threadIdx.x) % nx : 0;
#pragma unroll
            for (int r = 0; r < kPPT; ++r) {
                const int p = p0 + r * kBlock + threadIdx.x;
                if (r > 0 && two) {
                    ix += xstep;
                    if (ix >= nx) ix -= nx;
                }
                if (p < pend) {
                    const int lp = p - p0 + H;
                    const V u = stage[lp];
                    V xl, xr;
                    if (two) {
                        xl = stage[ix == 0 ? lp + nx - 1 : lp - 1];
                        xr = stage[ix == nx - 1 ? lp - nx + 1 : lp + 1];
                    } else {
                        xl = stage[lp - 1];
                        xr = stage[lp + 1];
                    }
                    const V yl = two ? stage[lp - nx] : zero, yr = two ? stage[lp + nx] : zero;
                    const V w = stencil_combine<T, V>(u, xl, xr, yl, yr, zero, zero, two ? 2 : 1, dg[r], tj, a0t,
                                                      a1t, a2t, sht);
                    wv[p] = w;
                    const float2 uf = dot_f2(u), wf = dot_f2(w);
                    const float2 vf = make_float2(tjf * uf.x, tjf * uf.y);
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        if (k < J) {
                            const float2 q = k == J - 1 ? uf : dot_f2(k == 0 ? q0[r] : (k == 1 ? q1[r] : q2[r]));
                            v[2 * k] = fmaf(q.x, vf.x, fmaf(q.y, vf.y, v[2 * k]));
                            v[2 * k + 1] = fmaf(q.x, vf.y, fmaf(-q.y, vf.x, v[2 * k + 1]));
                            v[8 + 2 * k] = fmaf(q.x, wf.x, fmaf(q.y, wf.y, v[8 + 2 * k]));
                            v[9 + 2 * k] = fmaf(q.x, wf.y, fmaf(-q.y, wf.x, v[9 + 2 * k]));
                        }
                    }
                }
            }
        }
        if (threadIdx.x == 0) sm.mphase = par;
        window_finish(sm, it, tb, J, v);
    }

    // Y prologue: every CTA of the item reduces X's partials and forms the
    // step's coefficients; the CTA owning tile 0 also stores the columns.
    static __device__ void dy_pro(Smem& sm, int item, const Runs& R, int j, bool last) {
        const EngineArgs& A = sm.A;
        const ItemDesc& it = A.item[item];
        ItemState* S = it.st;
        const int j0 = win_start(A, j);                                    // rows j0 .. j
        // the stored Hessenberg entries this step reads are loaded first, so
        // their latency overlaps the reduction below
        double2* Hw = sm.scratch;                                          // columns j0..j-2, pitch kHld
        const int ncol = max(0, j - 1 - j0);
        const bool hpre = ncol * kHld <= kBlock;
        double2 hreg = make_double2(0.0, 0.0), freg = make_double2(0.0, 0.0);
        if (hpre && threadIdx.x < ncol * kHld) {
            const int l = j0 + threadIdx.x / kHld, i = threadIdx.x - (threadIdx.x / kHld) * kHld;
            if (i <= l + 1) hreg = ldp(&S->H[l * (l + 3) / 2 + i]);
        }
        if (threadIdx.x < j) freg = ldp(((j - 1) & 1 ? S->hcol2 : S->hcol) + threadIdx.x);
        if (threadIdx.x <= j) {
            // s_i of the window's stored columns, t_j of the stored v_j
            sm.ssm[threadIdx.x] = threadIdx.x < j ? (threadIdx.x >= j0 ? ldd(&S->s[threadIdx.x]) : 1.0)
                                                  : ldp(&S->vt[j & 1]).x;
            if (threadIdx.x == j) sm.yscal[3] = ldp(&S->vt[j & 1]).y;                // 1/t_j
            if (threadIdx.x < j0) {
                sm.h1[threadIdx.x] = make_double2(0.0, 0.0);
                sm.h2[threadIdx.x] = make_double2(0.0, 0.0);
            }
        }
        __syncthreads();                                                   // scales s_i, t_j
        if (!last && j + 1 - j0 <= 16) {                                   // a_i, c and b_i, d together
            reduce_partials2(sm, it.part1, it.part2, it, R, j + 1 - j0, sm.ssm + j0, sm.h1 + j0, sm.h2 + j0);
        } else {
            reduce_partials<float>(sm, it.part1, it, R, j + 1 - j0, sm.ssm + j0, sm.h1 + j0);      // a_i, c
            if (!last) reduce_partials<float>(sm, it.part2, it, R, j + 1 - j0, sm.ssm + j0, sm.h2 + j0);  // b_i, d
        }
        if (hpre) {
            if (threadIdx.x < ncol * kHld) Hw[threadIdx.x] = hreg;
        } else {
            for (int t = threadIdx.x; t < ncol * kHld; t += kBlock) {
                const int l = j0 + t / kHld, i = t - (t / kHld) * kHld;
                if (i <= l + 1) Hw[t] = ldp(&S->H[l * (l + 3) / 2 + i]);
            }
        }
        if (threadIdx.x < j) sm.hfin[threadIdx.x] = freg;
        __syncthreads();
        // Thread i <= j finishes row i on its own (the window sums are recomputed
        // by every such thread): nu from one reciprocal square root, row i of
        // column j-1, row i of column j, and the sweep's coefficients.
        if (threadIdx.x <= j) {
            const int i = threadIdx.x;
            double aa2 = 0.0;
            double2 ab = make_double2(0.0, 0.0);                            // a^H b
            for (int l = j0; l < j; ++l) {
                const double2 a = sm.h1[l];
                aa2 += a.x * a.x + a.y * a.y;
                if (!last) ab = cfma(ab, cconj(a), sm.h2[l]);
            }
            const double nu2 = sm.h1[j].x - aa2;
            const double inv = nu2 > 0.0 ? rsqrt(nu2) : 0.0;
            const double nu = nu2 > 0.0 ? nu2 * inv : 0.0;
            double2 hf = make_double2(0.0, 0.0);                           // column j-1, row i
            if (j >= 1) {
                hf = i < j ? cadd(sm.hfin[i], sm.h1[i]) : make_double2(nu, 0.0);
                sm.hfin[i] = hf;
            }
            if (i == 0) {
                sm.yscal[0] = nu;
                sm.yscal[1] = sm.ssm[j] * inv;                              // s_j = t_j / nu
                sm.yscal[2] = inv;                                          // t_{j+1} = 1 / nu
            }
            if (!last) {
                double2 Ha = make_double2(0.0, 0.0);                        // (H a)_i over columns l < j
                for (int l = max(max(i - 1, 0), j0); l < j; ++l) {
                    const double2 Hil = l == j - 1 ? hf : Hw[(l - j0) * kHld + i];
                    Ha = cfma(Ha, Hil, sm.h1[l]);
                }
                double2 h;
                if (i < j0) h = make_double2(0.0, 0.0);                    // outside the window
                else if (i < j) h = cscale(csub(sm.h2[i], Ha), inv);
                else h = cscale(csub(cscale(csub(sm.h2[j], ab), inv), Ha), inv);
                sm.hnew[i] = h;
                const double2 gam = cadd(cscale(Ha, inv), h);
                // The sweep stores q_j and v_{j+1} unnormalised, with the scale
                // of each folded into its coefficients (no multiply per point):
                //   slot j   <- u_j - sum_i ca_i u_i,            q_j     = (t_j / nu) slot j,
                //   slot j+1 <- w - sum_i cg_i u_i - gq slot j,  v_{j+1} = (1 / nu) slot j+1,
                // u_i the stored window columns (q_i = s_i u_i), u_j = slot j, w = A v_j.
                if (i < j) {
                    const double2 ca = cscale(sm.h1[i], sm.ssm[i] * sm.yscal[3]);   // a_i s_i / t_j
                    sm.coef[i] = ca;
                    const double2 cg = cscale(gam, sm.ssm[i] * nu);                 // gamma_i s_i nu
                    sm.coefG[i] = cg;
                    if (sizeof(T) == 4) {                                   // rounded copies for a c64 basis
                        sm.coeff[i] = make_float2((float)ca.x, (float)ca.y);
                        sm.coefGf[i] = make_float2((float)cg.x, (float)cg.y);
                    }
                } else {
                    sm.ygq = cscale(gam, sm.ssm[j]);                                // gamma_j t_j
                }
            }
        }
        __syncthreads();
    }

    // Y sweep: q_j into slot j, v_{j+1} into slot j+1, by threads tid of nthr
    // (the whole CTA, or warps 1.. while warp 0 applies the rotations).
    static __device__ void dy(Smem& sm, int item, int tb, int te, int j, int tid, int nthr) {
        const ItemDesc& it = sm.A.item[item];
        const int it_n = it.n, it_tile = it.tile;
        const size_t n = (size_t)it_n;
        V* U = (V*)it.basis;
        V* uj = U + (size_t)j * n;
        V* wv = U + (size_t)(j + 1) * n;
        const V gq = cvt2<V>(sm.ygq);
        const int j0 = win_start(sm.A, j);
        if (tid == 0) {
            sm.nbytes += (unsigned long long)(run_points(it_n, it_tile, tb, te) * ((j - j0 + 4) * (long long)sizeof(V)));
            if (sizeof(T) == 8)
                sm.nflops += (unsigned long long)(run_points(it_n, it_tile, tb, te) * (16 * (j - j0) + 8));
        }
        for (int tile = tb; tile < te; ++tile) {
            const int p0 = tile * it_tile, pend = min(it_n, p0 + it_tile);
            for (int base = p0; base < pend; base += nthr * kChunk) {
                V qa[kChunk], va[kChunk];
#pragma unroll
                for (int r = 0; r < kChunk; ++r) {
                    const int p = base + r * nthr + tid;
                    qa[r] = p < pend ? ldv(uj + p) : mk2(T(0), T(0));
                    va[r] = p < pend ? ldv(wv + p) : mk2(T(0), T(0));
                }
#pragma unroll 2
                for (int q = j0; q < j; ++q) {
                    const V* uq = U + (size_t)q * n;
                    const V ca = coef_at<V>(sm, q), cg = coefg_at<V>(sm, q);
#pragma unroll
                    for (int r = 0; r < kChunk; ++r) {
                        const int p = base + r * nthr + tid;
                        const V u = p < pend ? ldv(uq + p) : mk2(T(0), T(0));
                        qa[r] = cfms(qa[r], ca, u);
                        va[r] = cfms(va[r], cg, u);
                    }
                }
#pragma unroll
                for (int r = 0; r < kChunk; ++r) {
                    const int p = base + r * nthr + tid;
                    if (p < pend) {
                        va[r] = cfms(va[r], gq, qa[r]);
                        uj[p] = qa[r];
                        wv[p] = va[r];
                    }
                }
            }
        }
    }

    // Y for a run of one tile swept by the whole CTA, with at most two older
    // vectors in the window: the sweep's loads (u_j, w and the window
    // vectors) are issued before the prologue, whose reduction and
    // coefficient recurrences then hide their latency.  The arithmetic is
    // the one of dy, in the same order.  Needs the register budget of one
    // CTA per SM (4 vectors x kPPT points per thread).
    static __device__ void dy_pre(Smem& sm, int item, const Runs& R, int tb, int j) {
        const ItemDesc& it = sm.A.item[item];
        const int it_n = it.n, it_tile = it.tile;
        const size_t n = (size_t)it_n;
        V* U = (V*)it.basis;
        V* uj = U + (size_t)j * n;
        V* wv = U + (size_t)(j + 1) * n;
        const int j0 = win_start(sm.A, j);
        const int nq = j - j0;                                  // 0, 1 or 2
        const int p0 = tb * it_tile, pend = min(it_n, p0 + it_tile);
        const V zero = mk2(T(0), T(0));
        V u[kPPT], w[kPPT], q0[kPPT], q1[kPPT];
#pragma unroll
        for (int r = 0; r < kPPT; ++r) {
            const int p = p0 + r * kBlock + threadIdx.x;
            const bool in = p < pend;
            u[r] = in ? ldv(uj + p) : zero;
            w[r] = in ? ldv(wv + p) : zero;
            q0[r] = (in && nq > 0) ? ldv(U + (size_t)j0 * n + p) : zero;
            q1[r] = (in && nq > 1) ? ldv(U + (size_t)(j0 + 1) * n + p) : zero;
        }
        dy_pro(sm, item, R, j, false);
        if (threadIdx.x == 0) {
            sm.nbytes += (unsigned long long)(run_points(it_n, it_tile, tb, tb + 1) * ((nq + 4) * (long long)sizeof(V)));
            if (sizeof(T) == 8)
                sm.nflops += (unsigned long long)(run_points(it_n, it_tile, tb, tb + 1) * (16 * nq + 8));
        }
        const V gq = cvt2<V>(sm.ygq);
        const V ca0 = nq > 0 ? coef_at<V>(sm, j0) : zero, cg0 = nq > 0 ? coefg_at<V>(sm, j0) : zero;
        const V ca1 = nq > 1 ? coef_at<V>(sm, j0 + 1) : zero, cg1 = nq > 1 ? coefg_at<V>(sm, j0 + 1) : zero;
#pragma unroll
        for (int r = 0; r < kPPT; ++r) {
            const int p = p0 + r * kBlock + threadIdx.x;
            V qa = u[r], va = w[r];
            if (nq > 0) {
                qa = cfms(qa, ca0, q0[r]);
                va = cfms(va, cg0, q0[r]);
            }
            if (nq > 1) {
                qa = cfms(qa, ca1, q1[r]);
                va = cfms(va, cg1, q1[r]);
            }
            va = cfms(va, gq, qa);
            if (p < pend) {
                uj[p] = qa;
                wv[p] = va;
            }
        }
    }

    // E2 prologue: y = R^{-1} g (back substitution, FP64), coefficients y_i s_i.
    static __device__ void e2_pro(Smem& sm, int item) {
        __syncthreads();                       // the previous run's sweep has read kk and basis
        const ItemDesc& it = sm.A.item[item];
        const ItemState* S = it.st;
        const int k = ldi(&S->k);
        const bool shared = ldi(&S->shared) != 0;
        const ItemDesc& src = shared ? sm.A.item[it.group] : it;   // owner of the basis used
        const int nR = k * (k + 1) / 2;
        double2* Rs = sm.scratch;
        for (int t = threadIdx.x; t < nR; t += kBlock) Rs[t] = ldp(&S->R[t]);
        if (threadIdx.x < k) {
            sm.gsm[threadIdx.x] = ldp(&S->g[threadIdx.x]);
            sm.ssm[threadIdx.x] = ldd(&src.st->s[threadIdx.x]);
        }
        if (threadIdx.x == 0) {
            sm.kk = k;
            sm.basis = src.basis;
            sm.xassign = shared && ldi(&S->cycles) == 1;
        }
        __syncthreads();
        if (threadIdx.x < 32) back_substitute(Rs, sm.gsm, sm.h2, k, sm.A.window);   // y_i into h2
        __syncthreads();
        if (threadIdx.x < k) {
            const double2 c = cscale(sm.h2[threadIdx.x], sm.ssm[threadIdx.x]);
            sm.coef[threadIdx.x] = c;
            sm.coeff[threadIdx.x] = make_float2((float)c.x, (float)c.y);
        }
        __syncthreads();
    }

    // E2: x += sum_i c_i u_i.  The correction is accumulated in the basis
    // precision (a cycle's correction is only accurate to the cycle's residual
    // reduction) and added to x in FP64.
    static __device__ void e2(Smem& sm, int item, int tb, int te) {
        const ItemDesc& it = sm.A.item[item];
        const int it_n = it.n, it_tile = it.tile;
        const size_t n = (size_t)it_n;
        const V* U = (const V*)sm.basis;
        double2* x = it.x;
        const int k = sm.kk;
        const bool assign = sm.xassign;                     // x not yet written (shared first cycle)
        acct(sm, run_points(it_n, it_tile, tb, te), k * (long long)sizeof(V) + 32);
        acctf(sm, run_points(it_n, it_tile, tb, te), (sizeof(T) == 8 ? 8 * k : 0) + 2);
        for (int tile = tb; tile < te; ++tile) {
            const int p0 = tile * it_tile, pend = min(it_n, p0 + it_tile);
            for (int r0 = 0; r0 < kPPT && p0 + r0 * kBlock < pend; r0 += kChunk) {
                V d[kChunk];
#pragma unroll
                for (int r = 0; r < kChunk; ++r) d[r] = mk2(T(0), T(0));
#pragma unroll 2
                for (int q = 0; q < k; ++q) {
                    const V* uq = U + (size_t)q * n;
                    const V c = coef_at<V>(sm, q);
#pragma unroll
                    for (int r = 0; r < kChunk; ++r) {
                        const int p = p0 + (r0 + r) * kBlock + threadIdx.x;
                        const V u = p < pend ? ldv(uq + p) : mk2(T(0), T(0));
                        d[r] = cfma(d[r], c, u);
                    }
                }
#pragma unroll
                for (int r = 0; r < kChunk; ++r) {
                    const int p = p0 + (r0 + r) * kBlock + threadIdx.x;
                    if (p < pend) x[p] = assign ? up2(d[r]) : cadd(ldv(x + p), up2(d[r]));
                }
            }
        }
    }
};

// E4 (one warp per item): true relative residual, decide, start a cycle.
__device__ void item_e4(const EngineArgs& A, int item, const Runs& R, const int* list, const int* prefix, int nl,
                        int ntasks) {
    const int lane = threadIdx.x & 31;
    const ItemDesc& it = A.item[item];
    ItemState* S = it.st;
    const int cycles = ldi(&S->cycles);
    double ss;
    if (cycles == 0 && A.mode == MODE_STEP && it.group >= 0) {
        // shared first cycle: ||b|| from the group item's partials (same b, same list)
        int lo = 0, hi = nl - 1;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (list[mid] < it.group) lo = mid + 1; else hi = mid;
        }
        ss = warp_norm_partials(A.item[it.group], item_runs(prefix, lo, ntasks));
    } else {
        ss = warp_norm_partials(it, R);
    }
    if (lane != 0) return;
    const double beta = sqrt(ss);
    double bnorm = cycles == 0 ? beta : ldd(&S->bnorm);
    if (cycles == 0) S->bnorm = beta;
    const double relres = bnorm > 0.0 ? beta / bnorm : 0.0;
    S->relres = relres;
    const int total = ldi(&S->total_iters);
    int status;
    if (it.is_group) {                              // shared Krylov basis of the members
        if (cycles == 0 && beta > 0.0 && beta <= 1e300) {
            S->s[0] = 1.0 / beta;
            S->vt[0] = make_double2(1.0 / beta, beta);
            S->k = 0;
            S->cycles = 1;
            S->total_iters = 0;
            status = ST_ARNOLDI;
        } else {
            status = ST_IDLE;
        }
        __threadfence();
        S->status = status;
        return;
    }
    if (!(beta <= 1e300) || !(bnorm <= 1e300) || !(relres <= 1e300)) {
        status = ST_FAILED;                         // NaN / Inf in the data
    } else if (bnorm == 0.0 || relres <= A.tol) {
        status = ST_CONVERGED;
    } else if (total >= A.max_iters) {
        status = ST_FAILED;
    } else {
        const bool shared = cycles == 0 && it.group >= 0;
        status = shared ? ST_SHARED : ST_ARNOLDI;
        S->shared = shared ? 1 : 0;
        S->s[0] = 1.0 / beta;
        S->vt[0] = make_double2(1.0 / beta, beta);
        S->g[0] = make_double2(beta, 0.0);
        S->k = 0;
        S->cycles = cycles + 1;
        S->cycle_tol_abs = fmax(A.tol * bnorm, A.inner_tol * beta);
    }
    if (status == ST_CONVERGED && cycles == 0 && A.mode == MODE_STEP && it.group >= 0) {
        S->k = 0;                                   // b = 0: x = 0, nothing to add (its x was not zeroed)
        S->ydone = 1;
        status = ST_DIRECT;
    }
    if (status == ST_CONVERGED || status == ST_FAILED || status == ST_DIRECT) {
        ItemStats* T = it.stats;
        T->iters += total;
        T->iters_sq += ldi(&S->sum_k2);
        T->cycles += cycles;
        T->max_sub_iters = max(T->max_sub_iters, total);
        T->resid = fmax(T->resid, relres);
        if (status == ST_FAILED) T->failed = 1;
    }
    __threadfence();
    S->status = status;
}

// P4 (one warp per item): Givens rotations of the new Hessenberg column.
__device__ void item_p4(const EngineArgs& A, int item, const Runs& R, int j) {
    const int lane = threadIdx.x & 31;
    const ItemDesc& it = A.item[item];
    ItemState* S = it.st;
    const double2 hl = lane <= j ? ldp(&S->hcol[lane]) : make_double2(0.0, 0.0);
    const double csl = lane < j ? ldd(&S->cs[lane]) : 0.0;
    const double2 snl = lane < j ? ldp(&S->sn[lane]) : make_double2(0.0, 0.0);
    const double ss = warp_norm_partials(it, R);
    const double hn = sqrt(ss);                  // h_{j+1,j} = ||w||
    double2 carry = shfl2(hl, 0);
    const int col = j * (j + 1) / 2;
    for (int i = 0; i < j; ++i) {
        const double2 b = shfl2(hl, i + 1);
        const double c = __shfl_sync(0xffffffffu, csl, i);
        const double2 s = shfl2(snl, i);
        const double2 nh = cfma(cscale(carry, c), s, b);
        carry = cfms(cscale(b, c), cconj(s), carry);
        if (lane == 0) S->R[col + i] = nh;
    }
    if (lane != 0) return;
    const double aa = sqrt(carry.x * carry.x + carry.y * carry.y);
    const double rr = sqrt(aa * aa + hn * hn);
    double c;
    double2 s, rjj;
    if (aa == 0.0) {
        c = 0.0;
        s = make_double2(1.0, 0.0);
        rjj = make_double2(hn, 0.0);
    } else {
        c = aa / rr;
        s = cscale(carry, hn / (aa * rr));
        rjj = cscale(carry, rr / aa);
    }
    const double2 gj = ldp(&S->g[j]);
    const double2 gj1 = cscale(cmul(cconj(s), gj), -1.0);
    S->R[col + j] = rjj;
    S->cs[j] = c;
    S->sn[j] = s;
    S->g[j] = cscale(gj, c);
    S->g[j + 1] = gj1;
    S->s[j + 1] = hn > 0.0 ? 1.0 / hn : 0.0;
    S->k = j + 1;
    const int total = ldi(&S->total_iters) + 1;
    S->total_iters = total;
    const double res = sqrt(gj1.x * gj1.x + gj1.y * gj1.y);
    const bool end = !(res > ldd(&S->cycle_tol_abs)) || j + 1 >= A.m || total >= A.max_iters ||
                     !(hn > 0.0) || !(rr > 0.0);
    if (end) S->sum_k2 = ldi(&S->sum_k2) + (j + 1) * (j + 1);
    __threadfence();
    S->status = end ? ST_CYCLE_END : ST_ARNOLDI;
}

// Cache the solution pointers and weights of problem `prob` in shared memory.
// With poles completed on the shared basis, yhat = sum_k alpha_k y_k over
// them (fixed order) and their x is not read.
__device__ void load_problem_items(Smem& sm, int prob) {
    const EngineArgs& A = sm.A;
    const ProblemDesc& pr = A.prob[prob];
    __syncthreads();                           // the previous problem's tiles are done with these
    const int nx = A.mode == MODE_BACKWARD ? 2 * pr.K : pr.K;
    for (int k = threadIdx.x; k < nx; k += kBlock) {
        const ItemDesc& it = A.item[pr.item0 + k];
        sm.xptr[k] = (A.mode == MODE_STEP && ldi(&it.st->status) == ST_DIRECT) ? nullptr : it.x;
    }
    for (int k = threadIdx.x; k < pr.K; k += kBlock) sm.alpha[k] = __ldg(pr.alpha + k);
    if (threadIdx.x == 0) sm.kyhat = 0;
    __syncthreads();
    if (threadIdx.x == 0) {
        int c = 0;
        for (int k = 0; k < nx; ++k) c += sm.xptr[k] != nullptr;
        sm.nxlive = c;
    }
    const int grp = A.mode == MODE_STEP ? A.item[pr.item0].group : -1;
    if (grp >= 0) {
        const ItemDesc& gd = A.item[grp];
        if (threadIdx.x < kMaxM) {
            const int i = threadIdx.x;
            double2 acc = make_double2(0.0, 0.0);
            int kmax = 0;
            for (int k = 0; k < pr.K; ++k) {
                if (sm.xptr[k] != nullptr) continue;
                const ItemState* M = A.item[pr.item0 + k].st;
                const int kk = ldi(&M->k);
                kmax = max(kmax, kk);
                if (i < kk) acc = cadd(acc, cmul(sm.alpha[k], ldp(&M->y[i])));
            }
            const double si = ldd(&gd.st->s[i]);
            sm.yhat[i] = cscale(acc, si);
            if (i == 0) {
                sm.kyhat = kmax;
                sm.gbasis = gd.basis;
            }
        }
        __syncthreads();
    }
}

// A pole whose residual estimate reaches the final tolerance on its group's
// shared basis during a step launch needs no x of its own: the pole sum takes
// alpha_k V y_k through the basis (sum_k alpha_k V y_k = V sum_k alpha_k y_k).
// Returns the status the member ends its shared cycle with.
__device__ __forceinline__ int member_end_status(const EngineArgs& A, const ItemDesc& md, ItemState* M,
                                                 double res, int total) {
    const double bnorm = ldd(&M->bnorm);
    // only an FP64 basis: the estimate of a c64 recurrence is not a residual bound
    if (A.mode != MODE_STEP || A.inner_tol > 0.0 || !(res <= A.tol * bnorm)) return ST_CYCLE_END;
    ItemStats* T = md.stats;
    T->iters += total;
    T->iters_sq += ldi(&M->sum_k2);
    T->cycles += ldi(&M->cycles);
    T->max_sub_iters = max(T->max_sub_iters, total);
    T->resid = fmax(T->resid, bnorm > 0.0 ? res / bnorm : 0.0);
    return ST_DIRECT;
}

// y = R^{-1} g of a pole completed on the shared basis (one warp; lane i holds
// row i, columns eliminated from the last).  Statuses stay as they are: every
// CTA builds its lists from them within the phase.
__device__ void member_direct_solve(const EngineArgs& A, int item) {
    const int lane = threadIdx.x & 31;
    ItemState* M = A.item[item].st;
    if (ldi(&M->ydone)) return;
    const int k = ldi(&M->k);
    double2 a0 = lane < k ? ldp(&M->g[lane]) : make_double2(0.0, 0.0);
    double2 a1 = lane + 32 < k ? ldp(&M->g[lane + 32]) : make_double2(0.0, 0.0);
    double2 y0 = make_double2(0.0, 0.0), y1 = make_double2(0.0, 0.0);
    // column l of R for rows lane and lane + 32, the next column fetched ahead
    // a windowed column l is zero above row l - L - 1 (those entries are not stored)
    auto col = [&](int l, double2& c0, double2& c1) {
        const double2* R = M->R + l * (l + 1) / 2;
        const int lo = A.window > 0 ? max(0, l - A.window - 1) : 0;
        c0 = (l >= 0 && lane <= l && lane >= lo) ? ldp(R + lane) : make_double2(0.0, 0.0);
        c1 = (l >= 0 && lane + 32 <= l && lane + 32 >= lo) ? ldp(R + lane + 32) : make_double2(0.0, 0.0);
    };
    // reciprocals of the diagonal, all rows at once (a division costs ~0.3 us)
    auto recip = [&](int i) {
        if (i >= k) return make_double2(0.0, 0.0);
        const double2 d = ldp(M->R + i * (i + 1) / 2 + i);
        const double den = d.x * d.x + d.y * d.y;
        return den > 0.0 ? cscale(cconj(d), 1.0 / den) : make_double2(0.0, 0.0);
    };
    const double2 inv0 = recip(lane), inv1 = recip(lane + 32);
    double2 c0, c1, n0, n1;
    col(k - 1, c0, c1);
    for (int l = k - 1; l >= 0; --l) {
        col(l - 1, n0, n1);
        double2 yl = make_double2(0.0, 0.0);
        if (lane == (l & 31)) {
            yl = l < 32 ? cmul(a0, inv0) : cmul(a1, inv1);
            if (l < 32) y0 = yl; else y1 = yl;
        }
        yl = shfl2(yl, l & 31);
        if (lane < l) a0 = csub(a0, cmul(c0, yl));
        if (lane + 32 < l) a1 = csub(a1, cmul(c1, yl));
        c0 = n0;
        c1 = n1;
    }
    if (lane < k) M->y[lane] = y0;
    if (lane + 32 < k) M->y[lane + 32] = y1;
    if (lane == 0) M->ydone = 1;
}

// P4 of a group (one warp, lane = member): every member's Hessenberg column is
// the group's column with its shift subtracted on the diagonal, because
// (B - s I) Q_j = Q_{j+1} (H_B - s [I; 0]) for the unshifted operator B; the
// members share the Krylov basis and keep their own rotations and residuals.
__device__ void group_p4(const EngineArgs& A, int gitem, const Runs& R, int j) {
    const int lane = threadIdx.x & 31;
    const ItemDesc& gd = A.item[gitem];
    ItemState* G = gd.st;
    const double hn = sqrt(warp_norm_partials(gd, R));
    const int col = j * (j + 1) / 2;
    const int nm = gd.nmembers;
    bool active = false;
    for (int mi = lane; mi < nm; mi += 32) {
        const ItemDesc& md = A.item[gd.member0 + mi];
        ItemState* S = md.st;
        if (ldi(&S->status) != ST_SHARED) continue;
        const double2 sh = md.shift;
        double2 carry = ldp(&G->hcol[0]);
        if (j == 0) carry = csub(carry, sh);
        for (int i = 0; i < j; ++i) {
            double2 b = ldp(&G->hcol[i + 1]);
            if (i + 1 == j) b = csub(b, sh);
            const double c = ldd(gd.gcs + (size_t)i * nm + mi);
            const double2 sn = ldp(gd.gsn + (size_t)i * nm + mi);
            const double2 nh = cfma(cscale(carry, c), sn, b);
            carry = cfms(cscale(b, c), cconj(sn), carry);
            S->R[col + i] = nh;
        }
        const double aa = sqrt(carry.x * carry.x + carry.y * carry.y);
        const double rr = sqrt(aa * aa + hn * hn);
        double c;
        double2 sn, rjj;
        if (aa == 0.0) {
            c = 0.0;
            sn = make_double2(1.0, 0.0);
            rjj = make_double2(hn, 0.0);
        } else {
            c = aa / rr;
            sn = cscale(carry, hn / (aa * rr));
            rjj = cscale(carry, rr / aa);
        }
        const double2 gj = ldp(&S->g[j]);
        const double2 gj1 = cscale(cmul(cconj(sn), gj), -1.0);
        gd.gcs[(size_t)j * nm + mi] = c;
        gd.gsn[(size_t)j * nm + mi] = sn;
        S->R[col + j] = rjj;
        S->g[j] = cscale(gj, c);
        S->g[j + 1] = gj1;
        S->k = j + 1;
        const int total = ldi(&S->total_iters) + 1;
        S->total_iters = total;
        const double res = sqrt(gj1.x * gj1.x + gj1.y * gj1.y);
        const bool end = !(res > ldd(&S->cycle_tol_abs)) || j + 1 >= A.m || total >= A.max_iters ||
                         !(hn > 0.0) || !(rr > 0.0);
        int stn = ST_SHARED;
        if (end) {
            S->sum_k2 = ldi(&S->sum_k2) + (j + 1) * (j + 1);
            stn = member_end_status(A, md, S, res, total);
        }
        __threadfence();
        S->status = stn;
        active = active || !end;
    }
    const bool any = __any_sync(0xffffffffu, active);
    if (lane == 0) {
        G->s[j + 1] = hn > 0.0 ? 1.0 / hn : 0.0;
        G->k = j + 1;
        __threadfence();
        G->status = any ? ST_ARNOLDI : ST_IDLE;
    }
}

// Complex Givens rotation that zeroes h against the (real, >= 0) subdiagonal
// hn: c = |a|/r, s = a hn/(|a| r), the new diagonal a r/|a| (a = carry,
// r = sqrt(|a|^2 + hn^2)); two reciprocal square roots instead of two square
// roots and three divisions.
__device__ __forceinline__ void givens(double2 a, double hn, double* c, double2* s, double2* rjj, double* r) {
    const double a2 = a.x * a.x + a.y * a.y;
    const double r2 = a2 + hn * hn;
    if (a2 == 0.0) {
        *c = 0.0;
        *s = make_double2(1.0, 0.0);
        *rjj = make_double2(hn, 0.0);
        *r = hn;
        return;
    }
    const double ia = rsqrt(a2), ir = rsqrt(r2);
    *c = a2 * ia * ir;                           // |a| / r
    *s = cscale(a, hn * ia * ir);
    *rjj = cscale(a, r2 * ir * ia);              // a r / |a|
    *r = r2 * ir;
}

// Delayed CGS2, step j: the CTA owning tile 0 of the item stores the completed
// column j-1 and the pending column j, and applies the Givens rotation of
// column j-1 (one warp; for a group, lane = member with its shifted column).
__device__ void dy_commit(const EngineArgs& A, Smem& sm, int item, int j, bool last, void* stage,
                          size_t stage_bytes) {
    const ItemDesc& it = A.item[item];
    ItemState* S = it.st;
    const double nu = sm.yscal[0];
    // a group's member rotations (column-major, i * nm + member) are copied to
    // shared memory by the whole CTA when they fit, so the serial loop below
    // does not wait on global loads
    // With a window, column j-1 is zero above row r0 = j-1-L, so the
    // rotations below i0 = r0-1 act on zeros: only rotations i0 .. j-2 run.
    const int jj = j - 1;                                            // column completed at this step
    const int i0 = A.window > 0 ? max(0, jj - A.window - 1) : 0;
    const int nmg = it.is_group ? it.nmembers : 0;
    const int nrot = jj > i0 ? nmg * (jj - i0) : 0;
    const bool staged = nrot > 0 && (size_t)nrot * (sizeof(double) + sizeof(double2)) <= stage_bytes;
    double2* st_sn = (double2*)stage;
    double* st_cs = (double*)(st_sn + nrot);
    if (staged) {
        const size_t base = (size_t)i0 * nmg;
        for (int t = threadIdx.x; t < nrot; t += kBlock) {
            st_sn[t] = ldp(it.gsn + base + t);
            st_cs[t] = ldd(it.gcs + base + t);
        }
        __syncthreads();
    }
    if (j >= 1 && threadIdx.x <= j) S->H[(j - 1) * (j + 2) / 2 + threadIdx.x] = sm.hfin[threadIdx.x];
    if (!last && threadIdx.x <= j) ((j & 1) ? S->hcol2 : S->hcol)[threadIdx.x] = sm.hnew[threadIdx.x];
    if (!last && threadIdx.x == 0) {                 // scales of the swept slots j and j + 1
        S->s[j] = sm.yscal[1];
        S->vt[(j + 1) & 1] = make_double2(sm.yscal[2], sm.yscal[0]);
    }
    if (threadIdx.x >= 32) return;
    const int lane = threadIdx.x;
    if (!it.is_group) {
        if (j == 0) {
            if (lane == 0) S->g[0] = cscale(ldp(&S->g[0]), nu);      // q_0 renormalised by nu
            return;
        }
        for (int i = i0 + lane; i < jj; i += 32) {
            sm.gcs_s[i] = ldd(&S->cs[i]);
            sm.gsn_s[i] = ldp(&S->sn[i]);
        }
        const int col = jj * (jj + 1) / 2;
        __syncwarp();
        if (lane != 0) return;
        // the state this commit reads is loaded before the serial rotations
        const double2 gj = ldp(&S->g[jj]);
        const int total = ldi(&S->total_iters) + 1;
        const double tola = ldd(&S->cycle_tol_abs);
        double2 carry = i0 == 0 ? sm.hfin[0] : make_double2(0.0, 0.0);
        for (int i = i0; i < jj; ++i) {
            const double2 b = sm.hfin[i + 1];
            const double c = sm.gcs_s[i];
            const double2 sn = sm.gsn_s[i];
            const double2 nh = cfma(cscale(carry, c), sn, b);
            carry = cfms(cscale(b, c), cconj(sn), carry);
            S->R[col + i] = nh;
        }
        const double hn = nu;
        double c, rr;
        double2 sn, rjj;
        givens(carry, hn, &c, &sn, &rjj, &rr);
        const double2 gj1 = cscale(cmul(cconj(sn), gj), -1.0);
        S->R[col + jj] = rjj;
        S->cs[jj] = c;
        S->sn[jj] = sn;
        S->g[jj] = cscale(gj, c);
        S->g[jj + 1] = gj1;
        S->k = j;
        S->total_iters = total;
        const bool end = !(res2_bound(A, gj1, j) > tola * tola) || last || total >= A.max_iters ||
                         !(hn > 0.0) || !(rr > 0.0);
        if (end) {
            S->sum_k2 = ldi(&S->sum_k2) + j * j;
            atomicAdd(A.epoch, 1u);                      // the Arnoldi list changes
        }
        S->status = end ? ST_CYCLE_END : ST_ARNOLDI;     // published by the phase barrier
        return;
    }
    // group: members' rotations of their shifted copies of column jj
    const int nm = it.nmembers;
    bool active = false;
    for (int mi = lane; mi < nm; mi += 32) {
        const ItemDesc& md = A.item[it.member0 + mi];
        ItemState* M = md.st;
        // every load of the member's state is issued before the serial rotations
        const int mstatus = ldi(&M->status);
        const double2 gj = ldp(&M->g[max(jj, 0)]);
        const int total = ldi(&M->total_iters) + 1;
        const double tola = ldd(&M->cycle_tol_abs);
        if (mstatus != ST_SHARED) continue;
        if (j == 0) {
            M->g[0] = cscale(gj, nu);
            active = true;
            continue;
        }
        const double2 sh = md.shift;
        double2 carry = i0 == 0 ? sm.hfin[0] : make_double2(0.0, 0.0);
        if (jj == 0) carry = csub(carry, sh);
        const int col = jj * (jj + 1) / 2;
        for (int i = i0; i < jj; ++i) {
            double2 b = sm.hfin[i + 1];
            if (i + 1 == jj) b = csub(b, sh);
            const size_t ri = (size_t)i * nm + mi;
            const size_t rs = (size_t)(i - i0) * nm + mi;
            const double c = staged ? st_cs[rs] : ldd(it.gcs + ri);
            const double2 sn = staged ? st_sn[rs] : ldp(it.gsn + ri);
            const double2 nh = cfma(cscale(carry, c), sn, b);
            carry = cfms(cscale(b, c), cconj(sn), carry);
            M->R[col + i] = nh;
        }
        const double hn = nu;
        double c, rr;
        double2 sn, rjj;
        givens(carry, hn, &c, &sn, &rjj, &rr);
        const double2 gj1 = cscale(cmul(cconj(sn), gj), -1.0);
        it.gcs[(size_t)jj * nm + mi] = c;
        it.gsn[(size_t)jj * nm + mi] = sn;
        M->R[col + jj] = rjj;
        M->g[jj] = cscale(gj, c);
        M->g[jj + 1] = gj1;
        M->k = j;
        M->total_iters = total;
        const double res2 = res2_bound(A, gj1, j);
        const bool end = !(res2 > tola * tola) || last || total >= A.max_iters || !(hn > 0.0) || !(rr > 0.0);
        int stn = ST_SHARED;
        if (end) {
            M->sum_k2 = ldi(&M->sum_k2) + j * j;
            stn = member_end_status(A, md, M, sqrt(res2), total);
        }
        M->status = stn;                                 // published by the phase barrier
        active = active || !end;
    }
    const bool any = __any_sync(0xffffffffu, active);
    if (lane == 0) {
        S->k = j;
        if (!(any && !last)) atomicAdd(A.epoch, 1u);     // the Arnoldi list changes
        S->status = (any && !last) ? ST_ARNOLDI : ST_IDLE;
    }
}

// PS: psi' = alpha_0 b + sum_k alpha_k x_k for one tile of a problem (poles
// completed on the shared basis enter as sum_i yhat_i u_i).
template <typename T>
__device__ void task_pole_sum(Smem& sm, int prob, int tile, int sub) {
    typedef typename C2<T>::t V;
    const ProblemDesc& pr = sm.A.prob[prob];
    const double2* b = step_in(sm.io, pr, prob, sub);
    double2* out = step_out(sm.io, pr, prob, sub);
    const int p0 = tile * kPsTile, pend = min(pr.n, p0 + kPsTile);
    acct(sm, pend - p0, 32 + 16 * (long long)sm.nxlive + (long long)sm.kyhat * (long long)sizeof(V));
    acctf(sm, pend - p0, 6 + 8 * ((long long)sm.nxlive + sm.kyhat));
    double2 acc[kPsPPT];
#pragma unroll
    for (int r = 0; r < kPsPPT; ++r) {
        const int p = p0 + r * kBlock + threadIdx.x;
        acc[r] = p < pend ? cmul(pr.alpha0, ldv(b + p)) : make_double2(0.0, 0.0);
    }
#pragma unroll 4
    for (int k = 0; k < pr.K; ++k) {
        const double2* xk = sm.xptr[k];
        if (xk == nullptr) continue;
        const double2 al = sm.alpha[k];
#pragma unroll
        for (int r = 0; r < kPsPPT; ++r) {
            const int p = p0 + r * kBlock + threadIdx.x;
            if (p < pend) acc[r] = cfma(acc[r], al, ldv(xk + p));
        }
    }
    const V* Ug = (const V*)sm.gbasis;
#pragma unroll 8
    for (int i = 0; i < sm.kyhat; ++i) {
        const V* ui = Ug + (size_t)i * pr.n;
        const double2 c = sm.yhat[i];
#pragma unroll
        for (int r = 0; r < kPsPPT; ++r) {
            const int p = p0 + r * kBlock + threadIdx.x;
            if (p < pend) acc[r] = cfma(acc[r], c, up2(ldv(ui + p)));
        }
    }
#pragma unroll
    for (int r = 0; r < kPsPPT; ++r) {
        const int p = p0 + r * kBlock + threadIdx.x;
        if (p < pend) out[p] = acc[r];
    }
}

// BA: adjoint accumulation for one tile of a problem (backward substep bs).
__device__ void task_adjoint(Smem& sm, int prob, int tile, int bs) {
    const ProblemDesc& pr = sm.A.prob[prob];
    const double2* gin = adj_in(sm.io, pr, prob, bs);
    double2* gout = adj_out(sm.io, pr, prob, bs);
    double* dV = sm.io.dLdV[prob];
    const int p0 = tile * kPsTile, pend = min(pr.n, p0 + kPsTile);
    acct(sm, pend - p0, 32 + 32 * (long long)pr.K + 16);
    acctf(sm, pend - p0, 6 + 20 * (long long)pr.K + 2);
    double2 g[kPsPPT];
    double dv[kPsPPT];
#pragma unroll
    for (int r = 0; r < kPsPPT; ++r) {
        const int p = p0 + r * kBlock + threadIdx.x;
        g[r] = p < pend ? cmul(cconj(pr.alpha0), ldv(gin + p)) : make_double2(0.0, 0.0);
        dv[r] = 0.0;
    }
#pragma unroll 2
    for (int k = 0; k < pr.K; ++k) {
        const double2* X = sm.xptr[k];
        const double2* Y = sm.xptr[pr.K + k];
        const double2 al = sm.alpha[k];
#pragma unroll
        for (int r = 0; r < kPsPPT; ++r) {
            const int p = p0 + r * kBlock + threadIdx.x;
            if (p < pend) {
                const double2 xv = ldv(X + p), yv = ldv(Y + p);
                g[r] = cfma(g[r], cconj(al), yv);
                dv[r] += cmul(al, cmul(cconj(yv), xv)).x;
            }
        }
    }
#pragma unroll
    for (int r = 0; r < kPsPPT; ++r) {
        const int p = p0 + r * kBlock + threadIdx.x;
        if (p < pend) {
            gout[p] = g[r];
            dV[p] += -pr.tau * dv[r];
        }
    }
}

// Contiguous share of the task range for this CTA.
__device__ __forceinline__ void my_range(int ntasks, int* s, int* e) {
    *s = (int)(((long long)blockIdx.x * ntasks) / gridDim.x);
    *e = (int)(((long long)(blockIdx.x + 1) * ntasks) / gridDim.x);
}

// MINB: CTAs per SM the register budget is sized for (FP64: 2 at 128
// registers, or 1 at up to 255 with wider update chunks; c64: 3).
template <typename T, int VG, int MINB>
__global__ void __launch_bounds__(kBlock, MINB) engine_kernel(const __grid_constant__ EngineArgs gA,
                                                            const __grid_constant__ IOArgs gio) {
    typedef Phases<T, VG, MINB> P;
    extern __shared__ __align__(16) int dyn[];
    __shared__ Smem sm;
    if (threadIdx.x == 0) {
        sm.A = gA;
        mbar_init(&sm.mbar, 1);
        sm.mphase = 0;
    }
    for (int q = threadIdx.x; q < kMaxBatch; q += kBlock) {
        sm.io.in[q] = gio.in[q];
        sm.io.out[q] = gio.out[q];
        sm.io.gout[q] = gio.gout[q];
        sm.io.dLdV[q] = gio.dLdV[q];
    }
    __syncthreads();
    const EngineArgs& A = sm.A;
    int* list = dyn;
    int* prefix = dyn + A.nitems;
    // tile staging buffer (16-byte aligned) after the list and prefix arrays
    typename C2<T>::t* ws = (typename C2<T>::t*)(dyn + ((2 * A.nitems + 2 + 3) & ~3));
    if (threadIdx.x == 0) sm.scratch = (double2*)ws;
    const int warp = threadIdx.x >> 5;
    const int gwarp = blockIdx.x * kWarps + warp;
    const int nwarps = gridDim.x * kWarps;
    // barrier counter; record 0 of both traces is the launch start
    __shared__ int tcount;
    if (threadIdx.x == 0) {
        tcount = 1;
        sm.nbytes = 0ull;
        sm.nflops = 0ull;
        const unsigned long long t0 = global_ns();
        if (A.trace != nullptr && blockIdx.x == 0 && A.trace_cap > 0) {
            A.trace[1] = 99ull;
            A.trace[2] = t0;
            A.trace[0] = 1ull;
        }
        if (A.cta_trace != nullptr && A.cta_trace_phases > 0 && (int)blockIdx.x < A.cta_trace_stride) {
            A.cta_trace[1 + blockIdx.x] = t0;
            if (blockIdx.x == 0) A.cta_trace[0] = 1ull;
        }
    }
    __syncthreads();

    for (int sub = 0; sub < A.max_sub; ++sub) {
        // substep start: every item of a live problem needs a first residual
        for (int i = blockIdx.x * kBlock + threadIdx.x; i < A.nitems; i += gridDim.x * kBlock) {
            const ItemDesc& it = A.item[i];
            ItemState* S = it.st;
            S->cycles = 0;
            S->total_iters = 0;
            S->sum_k2 = 0;
            S->shared = 0;
            S->k = 0;
            S->ydone = 0;
            S->status = sub < A.prob[it.problem].nsub ? ST_NEED_RES : ST_IDLE;
        }
        if (!phase_sync(A, TR_INIT, &tcount)) return;

        for (;;) {
            build_list(sm, list, prefix, (1u << ST_NEED_RES) | (1u << ST_CYCLE_END), true);
            if (sm.nl == 0) break;
            int s, e;
            my_range(sm.ntasks, &s, &e);
            for (int t = s; t < e;) {
                const int l = find_slot(prefix, sm.nl, t);
                const int te = min(prefix[l + 1], e) - prefix[l];
                P::e3(sm, sub, list[l], t - prefix[l], te);
                t = prefix[l] + te;
            }
            if (!phase_sync(A, TR_E3, &tcount)) return;
            for (int l = gwarp; l < sm.nl; l += nwarps)
                item_e4(A, list[l], item_runs(prefix, l, sm.ntasks), list, prefix, sm.nl, sm.ntasks);
            if (!phase_sync(A, TR_E4, &tcount)) return;

            for (int j = 0; A.ortho && j <= A.m; ++j) {             // delayed CGS2
                // the list changes only when a commit ends an item (epoch bump)
                if (threadIdx.x == 0) sm.ep_now = __ldcg(A.epoch);
                __syncthreads();
                if (j == 0 || sm.ep_now != sm.ep_seen) {
                    build_list(sm, list, prefix, 1u << ST_ARNOLDI);
                    if (threadIdx.x == 0) sm.ep_seen = sm.ep_now;
                }
                if (sm.nl == 0) break;
                const bool last = j == A.m;
                my_range(sm.ntasks, &s, &e);
                for (int t = s; t < e;) {
                    const int l = find_slot(prefix, sm.nl, t);
                    const int te = min(prefix[l + 1], e) - prefix[l];
                    P::dx(sm, ws, ws + kTile, list[l], t - prefix[l], te, j, !last);
                    t = prefix[l] + te;
                }
                if (!phase_sync(A, TR_DX, &tcount)) return;
                // Each item's commit (column store and rotations) runs on a CTA
                // without tiles when the task range leaves some (CTA b is then
                // idle rank b - s, and items go round-robin over the idle CTAs),
                // so the serial rotations share no SM with a sweep; otherwise on
                // the owner of the item's tile 0.
                const int nidle = sm.ntasks < (int)gridDim.x ? (int)gridDim.x - sm.ntasks : 0;
                for (int t = s; t < e;) {
                    const int l = find_slot(prefix, sm.nl, t);
                    const int te = min(prefix[l + 1], e) - prefix[l];
                    const int tb = t - prefix[l];
                    if (MINB == 1 && !last && !(tb == 0 && nidle == 0) && te - tb == 1 && j - win_start(A, j) <= 2) {
                        P::dy_pre(sm, list[l], item_runs(prefix, l, sm.ntasks), tb, j);
                        t = prefix[l] + te;
                        continue;
                    }
                    P::dy_pro(sm, list[l], item_runs(prefix, l, sm.ntasks), j, last);
                    if (tb == 0 && nidle == 0) {
                        // warp 0 applies the rotations while warps 1.. sweep this CTA's tiles
                        dy_commit(A, sm, list[l], j, last, ws, 2 * kTile * sizeof(*ws));
                        if (!last && threadIdx.x >= 32) P::dy(sm, list[l], tb, te, j, threadIdx.x - 32, kBlock - 32);
                        __syncthreads();
                    } else if (!last) {
                        P::dy(sm, list[l], tb, te, j, threadIdx.x, kBlock);
                    }
                    t = prefix[l] + te;
                }
                if (nidle > 0 && s == e) {
                    for (int l = (int)blockIdx.x - s; l < sm.nl; l += nidle) {
                        P::dy_pro(sm, list[l], item_runs(prefix, l, sm.ntasks), j, last);
                        dy_commit(A, sm, list[l], j, last, ws, 2 * kTile * sizeof(*ws));
                        __syncthreads();
                    }
                }
                if (!phase_sync(A, TR_DY, &tcount)) return;
            }
            for (int j = 0; !A.ortho && j < A.m; ++j) {             // CGS2
                build_list(sm, list, prefix, 1u << ST_ARNOLDI);
                if (sm.nl == 0) break;
                my_range(sm.ntasks, &s, &e);
                for (int t = s; t < e;) {
                    const int l = find_slot(prefix, sm.nl, t);
                    const int te = min(prefix[l + 1], e) - prefix[l];
                    P::p1(sm, ws, list[l], t - prefix[l], te, j);
                    t = prefix[l] + te;
                }
                if (!phase_sync(A, TR_P1, &tcount)) return;
                for (int t = s; t < e;) {
                    const int l = find_slot(prefix, sm.nl, t);
                    const int te = min(prefix[l + 1], e) - prefix[l];
                    P::p2_pro(sm, list[l], item_runs(prefix, l, sm.ntasks), j);
                    P::p2(sm, ws, list[l], t - prefix[l], te, j);
                    t = prefix[l] + te;
                }
                if (!phase_sync(A, TR_P2, &tcount)) return;
                for (int t = s; t < e;) {
                    const int l = find_slot(prefix, sm.nl, t);
                    const int te = min(prefix[l + 1], e) - prefix[l];
                    P::p3_pro(sm, list[l], item_runs(prefix, l, sm.ntasks), j);
                    P::p3(sm, list[l], t - prefix[l], te, j);
                    t = prefix[l] + te;
                }
                if (!phase_sync(A, TR_P3, &tcount)) return;
                for (int l = gwarp; l < sm.nl; l += nwarps) {
                    if (A.item[list[l]].is_group) group_p4(A, list[l], item_runs(prefix, l, sm.ntasks), j);
                    else item_p4(A, list[l], item_runs(prefix, l, sm.ntasks), j);
                }
                if (!phase_sync(A, TR_P4, &tcount)) return;
            }

            // poles completed on the shared basis: their y (one warp each)
            build_list(sm, list, prefix, 1u << ST_DIRECT);
            const bool direct = sm.nl > 0;
            for (int l = gwarp; l < sm.nl; l += nwarps) member_direct_solve(A, list[l]);
            __syncthreads();
            build_list(sm, list, prefix, 1u << ST_CYCLE_END);
            if (sm.nl > 0 || direct) {
                my_range(sm.ntasks, &s, &e);
                for (int t = s; t < e;) {
                    const int l = find_slot(prefix, sm.nl, t);
                    const int te = min(prefix[l + 1], e) - prefix[l];
                    P::e2_pro(sm, list[l]);
                    P::e2(sm, list[l], t - prefix[l], te);
                    t = prefix[l] + te;
                }
                if (!phase_sync(A, TR_E2, &tcount)) return;
            }
        }

        if (A.mode != MODE_SOLVE) {
            build_problem_list(sm, list, prefix, sub);
            int s, e;
            my_range(sm.ntasks, &s, &e);
            int cur = -1;
            for (int t = s; t < e; ++t) {
                const int l = find_slot(prefix, sm.nl, t);
                if (list[l] != cur) { cur = list[l]; load_problem_items(sm, cur); }
                if (A.mode == MODE_STEP) task_pole_sum<T>(sm, cur, t - prefix[l], sub);
                else task_adjoint(sm, cur, t - prefix[l], sub);
            }
            if (!phase_sync(A, TR_SUM, &tcount)) return;
        }
    }
    if (threadIdx.x == 0 && A.bytes != nullptr) {
        atomicAdd(A.bytes, sm.nbytes);
        atomicAdd(A.bytes + 1, sm.nflops);
    }
}

// ---- Chebyshev propagator (Sec. 4's comparison method) ---------------------------
//
// Clenshaw: b_{N+1} = b_{N+2} = 0, b_k = a_k u + 2 Ht b_{k+1} - b_{k+2}
// (k = N .. 1), out = a_0 u + Ht b_1 - b_2.  One grid barrier per degree: the
// stencil of b_{k+1} reads neighbours other CTAs wrote; b_k overwrites
// b_{k+2} in place (each point reads its own b_{k+2} only).

__global__ void __launch_bounds__(kBlock) cheb_kernel(const __grid_constant__ ChebArgs a) {
    const ProblemDesc& pr = *a.prob;
    const double* diag = pr.diag;
    const double a0 = pr.a[0], a1 = pr.a[1], a2 = pr.a[2];
    const double2 zero = make_double2(0.0, 0.0);
    const int gt = blockIdx.x * kBlock + threadIdx.x, gs = gridDim.x * kBlock;
    const int N = a.N, n = a.n;
    double2* X = a.b1;                       // b_{k+1}
    double2* Y = a.b2;                       // b_{k+2}, overwritten by b_k
    const double2 cN = __ldg(a.coef + N);
    for (int p = gt; p < n; p += gs) {
        X[p] = N > 0 ? cmul(cN, ldp(a.psi + p)) : zero;     // b_N (or 0 when N = 0)
        Y[p] = zero;                                        // b_{N+1}
    }
    if (!grid_sync(a.bar, a.err, a.timeout_ns)) return;
    const double s2 = 2.0 * a.scale;
    for (int k = N - 1; k >= 1; --k) {
        const double2 ck = __ldg(a.coef + k);
        for (int p = gt; p < n; p += gs) {
            const double2 h = stencil_apply<double, double2, false>(X, p, pr, diag, a0, a1, a2, zero);
            const double2 u = ldp(a.psi + p);
            const double2 y = ldp(Y + p);
            // b_k = c_k u + 2 Ht b_{k+1} - b_{k+2}, three fused multiply-adds per component
            Y[p] = make_double2(fma(s2, h.x, fma(ck.x, u.x, fma(-ck.y, u.y, -y.x))),
                                fma(s2, h.y, fma(ck.x, u.y, fma(ck.y, u.x, -y.y))));
        }
        double2* t = X;
        X = Y;
        Y = t;
        if (!grid_sync(a.bar, a.err, a.timeout_ns)) return;
    }
    const double2 c0 = __ldg(a.coef);
    for (int p = gt; p < n; p += gs) {
        const double2 u = ldp(a.psi + p);
        double2 r = cmul(c0, u);
        if (N > 0) {
            const double2 h = stencil_apply<double, double2, false>(X, p, pr, diag, a0, a1, a2, zero);
            const double2 y = ldp(Y + p);
            r = make_double2(r.x + a.scale * h.x - y.x, r.y + a.scale * h.y - y.y);
        }
        a.out[p] = r;
    }
    if (a.counters != nullptr && blockIdx.x == 0 && threadIdx.x == 0) {
        const int d = 1 + (pr.ny > 1) + (pr.nz > 1);
        const unsigned long long nn = (unsigned long long)n;
        // per degree: read b_{k+1} (stencil), u, b_{k+2} and the diagonal, write b_k
        atomicAdd(a.counters, nn * (16ull * 4 + 8ull) * (unsigned long long)(N > 0 ? N : 1) + nn * 32ull);
        atomicAdd(a.counters + 1, nn * (unsigned long long)(6 * d + 20) * (unsigned long long)(N > 0 ? N : 1));
    }
}

// ---- single-stage kernels ------------------------------------------------------

// w_k = A_k v_k for all poles (FP64): grid (ceil(n / kBlock), K).
__global__ void __launch_bounds__(kBlock) apply_kernel(const ProblemDesc* __restrict__ prob,
                                                       const ItemDesc* __restrict__ items,
                                                       const double2* __restrict__ v,
                                                       double2* __restrict__ w, int n) {
    const int p = blockIdx.x * kBlock + threadIdx.x;
    const int k = blockIdx.y;
    if (p >= n) return;
    const ProblemDesc& pr = *prob;
    const double2* vk = v + (size_t)k * n;
    w[(size_t)k * n + p] = stencil_apply<double, double2>(vk, p, pr, pr.diag, pr.a[0], pr.a[1], pr.a[2],
                                                          items[k].shift);
}

__global__ void __launch_bounds__(kBlock) pole_sum_kernel(const ProblemDesc* __restrict__ prob,
                                                          const double2* __restrict__ psi,
                                                          const double2* __restrict__ x,
                                                          double2* __restrict__ out, int n, int K) {
    const int p = blockIdx.x * kBlock + threadIdx.x;
    if (p >= n) return;
    const ProblemDesc& pr = *prob;
    double2 acc = cmul(pr.alpha0, psi[p]);
    for (int k = 0; k < K; ++k) acc = cadd(acc, cmul(pr.alpha[k], x[(size_t)k * n + p]));
    out[p] = acc;
}

}  // namespace

size_t engine_smem_bytes(int nitems, bool fp32, int ortho) {
    // list + prefix (ints, rounded to 16 bytes) + staging tiles of the basis type
    // (delayed CGS2 stages the v and w tiles of a step together)
    const size_t tiles = (ortho ? 2 : 1) * (size_t)kTile * (fp32 ? sizeof(float2) : sizeof(double2));
    return (size_t)((2 * nitems + 2 + 3) & ~3) * sizeof(int) +
           std::max(tiles, (size_t)kScratch * sizeof(double2));
}

static void* engine_fn(bool fp32, bool wide) {
    if (fp32) return (void*)engine_kernel<float, 32, 3>;
    return wide ? (void*)engine_kernel<double, 16, 1> : (void*)engine_kernel<double, 16, 2>;
}

int engine_max_grid(bool fp32, size_t smem, int device, bool wide) {
    void* fn = engine_fn(fp32, wide);
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(160 * 1024)) != cudaSuccess)
        return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, kBlock, smem) != cudaSuccess) return 0;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return 0;
    return nb * sms;
}

cudaError_t launch_engine(bool fp32, const EngineArgs& a, const IOArgs& io, int grid, size_t smem,
                          cudaStream_t stream, bool wide) {
    void* fn = engine_fn(fp32, wide);
    void* args[] = {(void*)&a, (void*)&io};
    return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kBlock), args, smem, stream);
}

cudaError_t launch_apply(const ProblemDesc* dprob, const ItemDesc* ditems, int K, const double2* v,
                         double2* w, int n, cudaStream_t stream) {
    dim3 grid((n + kBlock - 1) / kBlock, K);
    apply_kernel<<<grid, kBlock, 0, stream>>>(dprob, ditems, v, w, n);
    return cudaGetLastError();
}

cudaError_t launch_pole_sum(const ProblemDesc* dprob, const double2* psi, const double2* x, double2* out,
                            int n, int K, cudaStream_t stream) {
    pole_sum_kernel<<<(n + kBlock - 1) / kBlock, kBlock, 0, stream>>>(dprob, psi, x, out, n, K);
    return cudaGetLastError();
}

cudaError_t launch_cheb(const ChebArgs& args, int grid, cudaStream_t stream) {
    void* params[] = {(void*)&args};
    return cudaLaunchCooperativeKernel((const void*)cheb_kernel, dim3(grid), dim3(kBlock), params, 0, stream);
}

int cheb_max_grid(int device) {
    int per_sm = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cheb_kernel, kBlock, 0) != cudaSuccess) return -1;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return -1;
    return per_sm * sms;
}

}  // namespace rexi
