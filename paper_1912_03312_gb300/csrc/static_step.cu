// Allocation-free entry point: one rational evaluation of the engine with all
// of its workspace in a fixed, file-scope device array (see rexi.h,
// rexi_substep_static).  For callers that must not allocate device memory --
// code running inside an allocator callback, a host that pre-reserves all GPU
// memory for itself, or a sandbox that forbids cudaMalloc -- the workspace
// comes from this library's static image instead.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "../../include/rexi.h"
#include "engine.h"

using rexi::EngineArgs;
using rexi::IOArgs;
using rexi::ItemDesc;
using rexi::ItemState;
using rexi::ItemStats;
using rexi::ProblemDesc;

namespace {

// Every GPU that loads the library holds this array until the process exits.
constexpr size_t kStaticScratchBytes = (size_t)32 << 20;   // REXI_STATIC_SCRATCH_BYTES
static __device__ __align__(256) unsigned char g_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices];

// Device address of g_scratch on the current device, looked up once per device.
int scratch_address(int dev, unsigned char** out) {
    if (dev < 0 || dev >= kMaxDevices) return REXI_ECUDA;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return REXI_ECUDA;
        g_addr[dev] = p;
    }
    *out = (unsigned char*)g_addr[dev];
    return REXI_OK;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

__global__ void diag_kernel(const double* __restrict__ V, double* __restrict__ diag, float* __restrict__ diagf,
                            int n, double tau, double c, double sa) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        const double d = tau * (V[i] - c) - sa;
        diag[i] = d;
        diagf[i] = (float)d;
    }
}

}  // namespace

extern "C" int rexi_substep_static(const rexi_grid* g, const double* V, double tau, double c, int K,
                                   const double* z, const double* alpha, const double* alpha0,
                                   const rexi_options* opt_in, const void* psi_in, void* psi_out, void* stream,
                                   rexi_stats* st) {
    if (!g || !V || !z || !alpha || !alpha0 || !psi_in || !psi_out || !opt_in) return REXI_EINVAL;
    if (!(tau > 0.0) || !std::isfinite(tau) || !std::isfinite(c) || K < 1 || K > REXI_MAX_POLES) return REXI_EINVAL;
    if (g->ndim < 1 || g->ndim > 3 || !(g->hbar > 0.0) || !(g->mass > 0.0)) return REXI_EINVAL;
    const rexi_options opt = *opt_in;
    if (opt.precision != REXI_FP64 && opt.precision != REXI_MIXED) return REXI_EINVAL;
    if (opt.restart_m < 1 || opt.restart_m > REXI_MAX_RESTART || opt.max_iters < 1) return REXI_EINVAL;
    if (!(opt.tol > 0.0) || !std::isfinite(opt.tol) || !(opt.inner_tol >= 0.0) || !std::isfinite(opt.inner_tol))
        return REXI_EINVAL;
    if (opt.ortho != 0 && opt.ortho != 1) return REXI_EINVAL;
    if (opt.window == 0 && opt.restart_m > (opt.ortho == 1 ? REXI_MAX_RESTART_FULL : REXI_MAX_RESTART_FULL + 1))
        return REXI_EINVAL;
    if (opt.window < 0 || opt.window == 1 || opt.window > REXI_MAX_RESTART || (opt.window > 0 && opt.ortho != 1))
        return REXI_EINVAL;
    long long n = 1;
    int dims[3] = {1, 1, 1};
    double a[3] = {0.0, 0.0, 0.0};
    for (int d = 0; d < g->ndim; ++d) {
        if (g->n[d] < 1 || !(g->hi[d] > g->lo[d]) || !std::isfinite(g->hi[d] - g->lo[d])) return REXI_EINVAL;
        if (n > (1ll << 30) / g->n[d]) return REXI_EINVAL;   // checked before the product can overflow
        dims[d] = g->n[d];
        n *= g->n[d];
        const double h = (g->hi[d] - g->lo[d]) / g->n[d];
        a[d] = g->n[d] > 1 ? -tau * g->hbar * g->hbar / (2.0 * g->mass * h * h) : 0.0;
    }
    const bool fp32 = opt.precision == REXI_MIXED;
    const int m = opt.restart_m;
    const int ntiles = (int)((n + rexi::kTile - 1) / rexi::kTile);
    const int pv = 40;
    const size_t esz = fp32 ? sizeof(float2) : sizeof(double2);

    // Carve the workspace; reject what does not fit.
    size_t off = 0;
    auto take = [&](size_t bytes) { const size_t o = off; off = align256(off + bytes); return o; };
    const size_t o_bar = take(4 * sizeof(unsigned));
    const size_t o_prob = take(sizeof(ProblemDesc));
    const size_t o_items = take(sizeof(ItemDesc) * K);
    const size_t o_st = take(sizeof(ItemState) * K);
    const size_t o_stats = take(sizeof(ItemStats) * K);
    const size_t o_alpha = take(sizeof(double2) * K);
    const size_t o_diag = take(sizeof(double) * n);
    const size_t o_diagf = take(sizeof(float) * n);
    const size_t o_x = take(sizeof(double2) * n * K);
    const size_t o_basis = take(esz * n * (size_t)(m + 1) * K);
    const size_t o_p1 = take(sizeof(double2) * (size_t)ntiles * pv * K);
    const size_t o_p2 = take(sizeof(double2) * (size_t)ntiles * pv * K);
    const size_t o_pn = take(sizeof(double) * (size_t)ntiles * K);
    if (off > kStaticScratchBytes) return REXI_EINVAL;            // larger than the static workspace

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return REXI_ECUDA;
    unsigned char* base = nullptr;
    int r = scratch_address(dev, &base);
    if (r) return r;
    cudaStream_t s = (cudaStream_t)stream;

    ProblemDesc pr;
    std::memset(&pr, 0, sizeof(pr));
    pr.n = (int)n;
    pr.nx = dims[0];
    pr.ny = dims[1];
    pr.nz = dims[2];
    pr.ntiles = ntiles;
    pr.K = K;
    pr.item0 = 0;
    pr.nitems = K;
    pr.nsub = 1;
    for (int d = 0; d < 3; ++d) { pr.a[d] = a[d]; pr.af[d] = (float)a[d]; }
    pr.tau = tau;
    pr.alpha0 = make_double2(alpha0[0], alpha0[1]);
    pr.alpha = (const double2*)(base + o_alpha);
    pr.diag = (const double*)(base + o_diag);
    pr.diagf = (const float*)(base + o_diagf);

    ItemDesc items[REXI_MAX_POLES];
    std::memset(items, 0, sizeof(ItemDesc) * K);
    for (int k = 0; k < K; ++k) {
        ItemDesc& it = items[k];
        it.problem = 0;
        it.pole = k;
        it.group = -1;                                            // independent bases only
        it.is_group = 0;
        it.tile_off = k * ntiles;
        it.n = (int)n;
        it.ntiles = ntiles;
        it.tile = rexi::kTile;
        const double sr = z[2 * k] - tau * c, si = z[2 * k + 1];   // centred shift z_k - tau c
        it.shift = make_double2(sr, si);
        it.shiftf = make_float2((float)sr, (float)si);
        it.x = (double2*)(base + o_x) + (size_t)k * n;
        it.basis = base + o_basis + (size_t)k * (m + 1) * n * esz;
        it.st = (ItemState*)(base + o_st) + k;
        it.stats = (ItemStats*)(base + o_stats) + k;
        it.part1 = (double2*)(base + o_p1);
        it.part2 = (double2*)(base + o_p2);
        it.partn = (double*)(base + o_pn);
    }
    double2 al[REXI_MAX_POLES];
    for (int k = 0; k < K; ++k) al[k] = make_double2(alpha[2 * k], alpha[2 * k + 1]);

    // The array keeps the previous call's contents: reset what must start at zero.
    cudaError_t e = cudaMemsetAsync(base + o_bar, 0, 4 * sizeof(unsigned), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(base + o_stats, 0, sizeof(ItemStats) * K, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(base + o_prob, &pr, sizeof(pr), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(base + o_items, items, sizeof(ItemDesc) * K, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(base + o_alpha, al, sizeof(double2) * K, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return REXI_ECUDA;
    const double sa = 2.0 * (a[0] + a[1] + a[2]);
    diag_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(V, (double*)(base + o_diag), (float*)(base + o_diagf),
                                                            (int)n, tau, c, sa);
    if (cudaGetLastError() != cudaSuccess) return REXI_ECUDA;

    EngineArgs A;
    std::memset(&A, 0, sizeof(A));
    A.mode = rexi::MODE_STEP;
    A.nproblems = 1;
    A.nitems = K;
    A.m = m;
    A.max_iters = opt.max_iters;
    A.max_sub = 1;
    A.pv = pv;
    A.ortho = opt.ortho;
    A.window = opt.window;
    A.tol = opt.tol;
    A.inner_tol = fp32 ? opt.inner_tol : 0.0;
    A.timeout_ns = 4000000000ull;
    A.prob = (const ProblemDesc*)(base + o_prob);
    A.item = (const ItemDesc*)(base + o_items);
    A.bar = (unsigned*)(base + o_bar);
    A.epoch = (unsigned*)(base + o_bar) + 3;
    A.err = (int*)(base + o_bar) + 2;
    IOArgs io;
    std::memset(&io, 0, sizeof(io));
    io.in[0] = (const double2*)psi_in;
    io.out[0] = (double2*)psi_out;
    const size_t smem = rexi::engine_smem_bytes(K, fp32, A.ortho);
    const int maxg = rexi::engine_max_grid(fp32, smem, dev);
    if (maxg <= 0) return REXI_ECUDA;
    const int grid = std::max(1, std::min(maxg, K * ntiles));
    if (rexi::launch_engine(fp32, A, io, grid, smem, s) != cudaSuccess) return REXI_ECUDA;
    if (!st) return REXI_OK;

    ItemStats hs[REXI_MAX_POLES];
    int err = 0;
    e = cudaMemcpyAsync(&err, A.err, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hs, base + o_stats, sizeof(ItemStats) * K, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return REXI_ECUDA;
    std::memset(st, 0, sizeof(*st));
    st->n_sub = 1;
    bool failed = false;
    for (int k = 0; k < K; ++k) {
        st->iters[k] = hs[k].iters;
        st->cycles[k] = hs[k].cycles;
        st->iters_sq[k] = hs[k].iters_sq;
        st->resid[k] = hs[k].resid;
        st->total_iters += hs[k].iters;
        st->total_cycles += hs[k].cycles;
        st->max_iters_seen = std::max(st->max_iters_seen, hs[k].max_sub_iters);
        failed = failed || hs[k].failed;
    }
    st->status = err ? err : (failed ? REXI_ENOCONV : REXI_OK);
    return st->status;
}
