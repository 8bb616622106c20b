// Shared-basis Lanczos path of the engine (host/device descriptor).
//
// All K shifted systems (tau H - z_k I) x_k = psi of one rational evaluation
// (Eq. (5)) share one Krylov space K_m(B, psi), B = tau (H - c) (Sec. 5: the
// spaces of shifted systems coincide).  B is real symmetric, so the basis obeys
// a three-term recurrence with real coefficients; every pole keeps its own
// Givens QR of the tridiagonal T_k - s_k [I; 0] (s_k = z_k - tau c) and stops on
// a rigorous bound of its true residual.  One persistent cooperative launch
// runs all substeps; one grid barrier per Krylov step.
#pragma once

#include <cuda_runtime.h>

#include "engine.h"

namespace rexi {

constexpr int kLzBlock = 256;          // threads per CTA
constexpr int kLzMaxM = 512;           // largest Krylov dimension per substep
constexpr int kLzMaxInterior = 2048;   // interior points of one tile
constexpr int kLzMaxExt = 4096;        // tile plus its halo

enum : int { LZ_STEP = 0, LZ_SOLVE = 1 };

// trace codes (after the phase codes of the engine)
enum : int { TR_LZ_SWEEP = 11, TR_LZ_SOLVE = 12, TR_LZ_SUM = 13 };

// Sites of the index checks of a build with REXI_DEBUG defined (the numbers a
// failed check records; 0 = none).
enum : int {
    LZ_SITE_SMEM = 1,        // shared-memory layout of the launch, tile boxes
    LZ_SITE_STAGE = 2,       // copies into shared memory (extended box, diagonal)
    LZ_SITE_STAGE_SRC = 3,   // their global sources
    LZ_SITE_RING = 4,        // halo ring list of a resident tile
    LZ_SITE_BASIS = 5,       // basis vectors (stores of phase A, reads of the final pass)
    LZ_SITE_STENCIL = 6,     // stencil and diagonal reads of phase B
    LZ_SITE_WT = 7,          // B u stores
    LZ_SITE_PART = 8,        // per-CTA partial sums
    LZ_SITE_ROWS = 9,        // rows of R (stores, staging for the back substitution)
    LZ_SITE_Y = 10,          // y_k, coefficients and scales of the final pass
    LZ_SITE_STATE = 11,      // input, output and substep states
    LZ_SITE_COUNT = 12
};

struct LzArgs {
    int mode;                  // LZ_STEP: nsub substeps ending in the pole sum; LZ_SOLVE: x_k for every pole
    int n, nx, ny, nz;         // grid (x fastest); unused dimensions have extent 1
    int K;                     // poles
    int nsub;                  // substeps (1 in LZ_SOLVE)
    int m;                     // largest Krylov dimension (columns) per substep
    double a[3];               // stencil coefficients -tau hbar^2/(2 m h_d^2); 0 for extent-1 dimensions
    double fold;               // f = |a_d| of the first nonzero a_d (1 if none); the kernel stores w' = B u / f
    double ratio[3];           // a_d / f (-1 for that first dimension)
    int unit_ok;               // 1: the recurrence may run unscaled (||B|| / f <= 2^16)
    const double* diag;        // [n] (tau (V - c) - 2 sum_d a_d) / f
    const float2* diag_df;     // [n] the same diagonal as double-float pairs (hi, lo)
    int df;                    // 1: the recurrence from sweep 1 on in double-float on the FP32 pipe
    const double2* shift;      // [K] centred shifts s_k = z_k - tau c
    const double2* alpha;      // [K] weights
    double2 alpha0;
    double tol;                // per-pole stop: bound of ||b - A_k x_k|| <= tol ||b||
    int stage_rows;            // rows of R the control CTA stages per chunk (fit the dynamic shared memory)
    int tx, ty, tz;            // tile box
    int gx, gy, gz;            // tiles per dimension
    int ntiles;
    int resident;              // 1: at most one tile per CTA, its state kept in shared memory between sweeps
    const double2* in;         // LZ_STEP: psi_in; LZ_SOLVE: right-hand side b
    double2* out;              // LZ_STEP: psi_out; LZ_SOLVE: x [K][n]
    double2* tmp0;             // substep states (ping-pong)
    double2* tmp1;
    double2* basis;            // [m + 2][n]: u_1 .. u_{m+2} (u_0 is the substep's input state); resident
                               // tiles or df: each entry the double-float pairs (re_hi, re_lo, im_hi, im_lo)
    double2* wt;               // [2][n]: B u_j by parity of j
    float4* part;              // [2][grid]: per-CTA partial sums (||u_j||^2, Re u_j^H B u_j) as double-float pairs
    double2* rows;             // [m][K][3]: scaled rows of every pole's R for the back substitution
    double2* ybuf;             // [m][K]: y_k of the last substep (LZ_STEP) / unused
    double2* coef;             // LZ_STEP: [m] coefficients of u_r in psi'; LZ_SOLVE: [K][m]
    double* rho;               // [m + 2]: scale of every stored vector (q_j = rho_j u_j)
    int* stop;                 // [nsub]: columns of substep s once every pole has stopped (-1 before)
    int* cols;                 // [2 nsub]: columns and Krylov sweeps of every substep
    ItemStats* stats;          // [K] per pole (zeroed before the launch)
    unsigned* bar;             // [2] grid barrier (zeroed before the launch)
    int* err;                  // sticky error word
    unsigned long long timeout_ns;
    unsigned long long* trace; // optional [1 + 2 cap]: (phase, ns) at every barrier
    int trace_cap;
    unsigned long long* bytes; // [3]: algorithmic bytes, FP64 flops and FP32-pipe operations of the launch
                               // (added by the control CTA)
    int part_cap;              // slots per parity of part (>= ncta)
    int cta0, ncta;            // the CTAs of the launch that work for this problem
    long long* dbg;            // REXI_DEBUG builds: [4] first failed check (site, index, extent), count
    int dbg_trip;              // REXI_DEBUG builds: a site whose every check fails (0: none)
};

// Input and output states of a batched launch (problem p: in[p], out[p]).
struct LzIO {
    const double2* in[kMaxBatch];
    double2* out[kMaxBatch];
};

cudaError_t launch_lanczos(const LzArgs& args, int grid, size_t smem, cudaStream_t stream);
// Several problems in one cooperative launch: d_args[p] (device) describes
// problem p with its CTA range; d_cta_prob[c] (device) is the problem of CTA c.
cudaError_t launch_lanczos_batched(const LzArgs* d_args, const unsigned char* d_cta_prob, const LzIO& io, int grid,
                                   size_t smem, cudaStream_t stream);
// Zero the barrier, error, work and statistics words and clear the stop words
// of the B problems of d_args (device), before a batched launch.
cudaError_t lanczos_reset(const LzArgs* d_args, int B, cudaStream_t stream);
int lanczos_max_grid(size_t smem, int device, bool batched = false);   // co-resident CTAs (<= 0: error)
size_t lanczos_smem_bytes(int tx, int ty, int tz, int hx, int hy, int hz, bool resident);
size_t lanczos_static_smem();                       // static shared memory of the kernel (0: error)

}  // namespace rexi
