// Device-side descriptors of the persistent REXI engine (shared by the kernel
// translation unit and the host API).
#pragma once

#include <cuda_runtime.h>

namespace rexi {

constexpr int kBlock = 256;            // threads per CTA
constexpr int kPPT = 8;                // points per thread per task
constexpr int kTile = kBlock * kPPT;   // points per (item, tile) task
constexpr int kMaxM = 64;              // largest restart length (windowed bases; full ones: 31 / 32)
constexpr int kHld = kMaxM + 2;        // pitch of Hessenberg columns staged in shared memory
constexpr int kScratch = kMaxM * (kMaxM + 3) / 2;   // shared scratch entries (R or H columns)
constexpr int kMaxItems = 4096;        // items (shifted solves) per launch
constexpr int kMaxBatch = 128;         // problems per launch
constexpr int kMaxPoles = 256;         // poles per problem

// item status values
enum : int {
    ST_NEED_RES = 0,   // FP64 residual (refinement) due
    ST_ARNOLDI = 1,    // inside an Arnoldi cycle
    ST_CYCLE_END = 2,  // cycle finished: x update due
    ST_CONVERGED = 3,
    ST_FAILED = 4,
    ST_IDLE = 5,       // not part of the current substep
    ST_SHARED = 6,     // pole in its first cycle on its group's shared Krylov basis
    ST_DIRECT = 7,     // converged on the shared basis in a step launch: its V y joins the
                       // pole sum through the group's basis (y computed once, see ydone)
};

// kernel modes
enum : int {
    MODE_STEP = 0,       // substeps of Eq. (5): solves + pole sum
    MODE_SOLVE = 1,      // one set of solves, x left in the item buffers
    MODE_BACKWARD = 2,   // adjoint substeps: 2K solves + adjoint accumulation
};

struct ProblemDesc {
    int n, nx, ny, nz;
    int ntiles;
    int K;               // poles of this problem (items per substep: K, or 2K backward)
    int item0;           // first item of this problem in the launch
    int nitems;          // items of this problem
    int nsub;            // substeps to run
    int pad0;
    double a[3];         // stencil coefficients -tau hbar^2 / (2 m h_d^2) (0 for unused dims)
    float af[3];
    float pad1;
    double tau;
    double2 alpha0;
    const double2* alpha;      // device [K]
    const double* diag;        // device [n]: tau (V - c) - 2 sum_d a_d
    const float* diagf;        // device [n], float copy (mixed precision)
    double2* tmp0;             // ping-pong state buffer (c128)
    double2* tmp1;             // ping-pong state buffer (c128)
    double2* ckpt;             // backward: [nsub][n] forward states (ckpt[0] unused)
};

// Per-call buffers, passed by value in the kernel parameters.
struct IOArgs {
    const double2* in[kMaxBatch];     // step input / solve rhs / psi_n (backward)
    double2* out[kMaxBatch];          // step output / grad_in (backward)
    const double2* gout[kMaxBatch];   // backward: G at the step output
    double* dLdV[kMaxBatch];          // backward: accumulated gradient
};

struct ItemDesc {
    int problem;
    int pole;            // pole index k
    int adjoint;         // 1: solve with conj shift against the adjoint state
    int tile_off;        // first tile of this item in the partial buffers
    int n;               // points of the item's problem
    int ntiles;          // tiles of this item (ceil(n / tile))
    int tile;            // points per tile: a multiple of kBlock, at most kTile
    double2 shift;       // A = stencil + diag - shift
    float2 shiftf;
    double2* x;          // c128 [n]
    void* basis;         // T2 [m+1][n]
    int group;           // pole items: item index of the shared-cycle group, -1 if none
    int is_group;        // 1: group item (Arnoldi on the unshifted operator for its members)
    int member0;         // group items: first member item index
    int nmembers;        // group items: number of members
    double* gcs;         // group items: Givens cosines [kMaxM][nmembers]
    double2* gsn;        // group items: Givens sines   [kMaxM][nmembers]
    struct ItemState* st;
    struct ItemStats* stats;
    double2* part1;      // [tiles][pv] partial dots, first CGS pass
    double2* part2;      // [tiles][pv] partial dots, second CGS pass
    double* partn;       // [tiles] partial squared norms
};

struct ItemState {
    int status, k, total_iters, cycles;
    int sub_iters, sub_cycles, sum_k2, shared;
    int ydone, pad_y;                      // ST_DIRECT: y computed
    double bnorm, beta, cycle_tol_abs, relres;
    double s[kMaxM + 1];                   // scales of the stored columns (column i = s_i x slot i);
                                           // s[0] = 1/beta at a cycle's start
    double2 vt[2];                         // delayed CGS2: (t_j, 1/t_j) of the stored v_j (v_j = t_j x
                                           // slot j), by parity of j
    double cs[kMaxM];
    double2 sn[kMaxM];
    double2 g[kMaxM + 1];
    double2 hcol[kMaxM + 1];               // pending column (CGS2; delayed CGS2: even steps)
    double2 hcol2[kMaxM + 1];              // delayed CGS2: pending column of odd steps
    double2 R[kMaxM * (kMaxM + 1) / 2];    // packed upper triangle, column j at j(j+1)/2
    double2 H[kMaxM * (kMaxM + 3) / 2];    // unrotated Hessenberg, column l (l+2 entries) at l(l+3)/2
    double2 y[kMaxM];                      // ST_DIRECT poles: least-squares solution on the shared basis
};

// Per-call statistics of one item (zeroed before every launch).
struct ItemStats {
    int iters, cycles, failed, max_sub_iters;
    double resid;
    int iters_sq, pad;        // sum over cycles of (cycle length)^2
};

struct EngineArgs {
    int mode;
    int nproblems;
    int nitems;
    int m;               // restart length
    int max_iters;
    int max_sub;         // largest nsub over problems
    int pv;              // pitch of the partial buffers (>= m + 1)
    int ortho;           // 0: CGS2 (two reductions per step), 1: delayed CGS2 (one reduction)
    double tol;          // relative residual target
    double inner_tol;    // relative reduction per cycle (mixed), 0 = none
    unsigned long long timeout_ns;
    const ProblemDesc* prob;
    const ItemDesc* item;
    unsigned* bar;       // [2]: arrivals, completed barriers (zeroed before every launch)
    unsigned* epoch;     // bumped when an Arnoldi item leaves the Arnoldi state (list rebuilds)
    int* err;            // sticky error word
    unsigned long long* trace;   // optional: [1 + 2*cap] (count, then (phase, ns) pairs)
    int trace_cap;
    unsigned long long* cta_trace;   // optional: [1 + phases*stride] arrival ns of every CTA at every barrier
    int cta_trace_phases;
    int cta_trace_stride;
    int window;          // delayed CGS2: 0 = whole basis; L = only the last L vectors (Hermitian operators)
    int pad3;
    unsigned long long* bytes;   // optional [2]: algorithmic bytes and FP64 flops of the launch (atomic sums)
};

// phase codes recorded in the trace at the barrier that ends each phase
enum : int { TR_INIT = 0, TR_E3 = 1, TR_E4 = 2, TR_P1 = 3, TR_P2 = 4, TR_P3 = 5, TR_P4 = 6, TR_E2 = 7,
             TR_SUM = 8, TR_DX = 9, TR_DY = 10 };

// Chebyshev propagator of the comparison method of Sec. 4, evaluated with the
// Clenshaw recurrence on the plan's FP64 operator B = tau (H - c):
// Ht = scale B has its spectrum in [-1, 1]; out = sum_k coef_k T_k(Ht) psi.
struct ChebArgs {
    const ProblemDesc* prob;     // the plan's problem descriptor (stencil of B, FP64 diagonal)
    const double2* psi;          // input, [n]
    double2* out;                // result, [n] (may alias psi)
    double2* b1;                 // Clenshaw buffers, [n] each
    double2* b2;
    const double2* coef;         // [N + 1]: a_k exp(-i dt c / hbar)
    int N;
    int n;
    double scale;                // 1 / (tau W)
    unsigned* bar;               // [2] grid barrier: arrivals, completed barriers (zeroed per launch)
    int* err;
    unsigned long long timeout_ns;
    unsigned long long* counters;   // optional [2]: algorithmic bytes, FP64 flops
};
cudaError_t launch_cheb(const ChebArgs& args, int grid, cudaStream_t stream);
int cheb_max_grid(int device);   // co-resident CTAs of the Chebyshev kernel (<= 0: error)

// Launch the persistent kernel; T = float (mixed) or double (fp64).  wide
// (FP64 only): the instantiation for one CTA per SM (up to 255 registers,
// 8-point update chunks); its largest co-resident grid is one CTA per SM.
cudaError_t launch_engine(bool fp32_basis, const EngineArgs& args, const IOArgs& io, int grid,
                          size_t smem, cudaStream_t stream, bool wide = false);
int engine_max_grid(bool fp32_basis, size_t smem, int device, bool wide = false);
size_t engine_smem_bytes(int nitems, bool fp32, int ortho);

// Single-stage kernels.
cudaError_t launch_apply(const ProblemDesc* dprob, const ItemDesc* ditems, int K, const double2* v,
                         double2* w, int n, cudaStream_t stream);
cudaError_t launch_pole_sum(const ProblemDesc* dprob, const double2* psi, const double2* x,
                            double2* out, int n, int K, cudaStream_t stream);

}  // namespace rexi
