// C ABI of the REXI engine (declared in include/rexi.h): plan construction on
// the host (Sec. 3.1-3.3 of Rittich & Speck, arXiv:1912.03312), device
// workspace, and the launches of the persistent engine.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <complex>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "../../include/rexi.h"
#include "engine.h"
#include "fcf.h"
#include "lanczos.h"

using rexi::EngineArgs;
using rexi::IOArgs;
using rexi::ItemDesc;
using rexi::ItemState;
using rexi::ItemStats;
using rexi::ProblemDesc;
typedef std::complex<double> cd;

namespace {

constexpr unsigned long long kTimeoutNs = 4000000000ull;   // 4 s per barrier wait

struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
};

// One descriptor set: a problem descriptor and its items on the device.
struct DescSet {
    ProblemDesc* d_prob = nullptr;
    ItemDesc* d_items = nullptr;
    int nitems = 0;
    int ntiles_items = 0;
};

}  // namespace

struct rexi_plan {
    int device = 0;
    rexi_grid grid{};
    rexi_options opt{};
    int n = 0, K = 0, m = 30, n_sub = 1;
    int dims[3] = {1, 1, 1};
    double h[3] = {1, 1, 1};
    double dt = 0, tau = 0, R1 = 0, E_min = 0, E_max = 0, c = 0, W = 0, tol = 0;
    bool fp32 = true;
    rexi::FcfResult fcf;
    std::vector<cd> z, alpha;
    cd alpha0 = 0.0;
    double a[3] = {0, 0, 0};
    std::vector<double> V;                       // host copy of the potential
    int ntiles = 0, pv = 32;
    int tile_pole = rexi::kTile;                 // points per tile of pole items
    int tile_group = rexi::kBlock * 2;           // points per tile of shared-cycle group items
    int max_tiles = 0;                           // partial-buffer slots per item (256-point tiles)
    int ctas_per_sm = 0;                         // 0: as many as fit
    unsigned long long timeout_ns = kTimeoutNs;  // limit of every device-side wait
    int warn = REXI_OK;
    // device memory
    std::vector<void*> allocs;
    double* d_diag = nullptr;
    float* d_diagf = nullptr;
    double2* d_alpha = nullptr;
    double2* d_tmp0 = nullptr;
    double2* d_tmp1 = nullptr;
    double2* d_hin = nullptr;                    // staging for rexi_step_host
    double2* d_hout = nullptr;
    unsigned* d_bar = nullptr;
    int* d_err = nullptr;
    unsigned long long* d_bytes = nullptr;       // [3] algorithmic bytes, FP64 flops, FP32-pipe ops of the last launch
    double2* d_cheb = nullptr;                   // Chebyshev coefficients (rexi_cheb_step)
    int cheb_cap = 0;
    int nit_cap = 0;                             // pole items with workspace (K or 2K)
    int ngroups = 0;                             // shared-cycle group items (0, 1 or 2)
    bool shared = true;
    double* d_gcs = nullptr;                     // group Givens cosines [ngroups][kMaxM][K]
    double2* d_gsn = nullptr;
    double2* d_x = nullptr;
    void* d_basis = nullptr;
    ItemState* d_st = nullptr;
    ItemStats* d_stats = nullptr;
    double2* d_part1 = nullptr;
    double2* d_part2 = nullptr;
    double* d_partn = nullptr;
    double2* d_ckpt = nullptr;
    DescSet fwd, one, bwd;
    // engine settings of the general (item) engine; a Lanczos plan uses it only
    // for the calls the Lanczos kernel does not cover (adjoint, single stages)
    int eng_ortho = 1, eng_window = 0;
    // shared-basis Lanczos path (opt.ortho == 2)
    bool lanczos = false;
    int lz_m = 0;                                // largest Krylov dimension per substep
    int lz_tx = 1, lz_ty = 1, lz_tz = 1;         // tile box
    int lz_cps = 2;                              // CTAs per SM
    int lz_target = 0;                           // largest interior points per tile (0: choose)
    int lz_grid = 0, lz_stage = 1;
    bool lz_resident = false;                    // one tile per CTA, state kept in shared memory
    size_t lz_smem = 0;
    int lz_part_cap = 0;                         // CTAs the partial buffer holds
    double2* d_lz_basis = nullptr;
    double2* d_lz_wt = nullptr;
    float4* d_lz_part = nullptr;
    double2* d_lz_rows = nullptr;
    double2* d_lz_ybuf = nullptr;
    double2* d_lz_coef = nullptr;
    double* d_lz_rho = nullptr;
    int* d_lz_stop = nullptr;
    int* d_lz_cols = nullptr;
    double2* d_lz_shift = nullptr;
    double* d_lz_diag = nullptr;                 // diagonal divided by the stencil fold factor
    float2* d_lz_diagdf = nullptr;               // the same as double-float pairs (REXI_DF64)
    long long* d_dbg = nullptr;                  // index-check builds: record of the last Lanczos launch
    int dbg_trip = 0;                            // index-check builds: site made to fail
    double lz_fold = 1.0;
    ProblemDesc hprob{};                         // forward problem descriptor (host copy)
    int last_status = REXI_OK;
    int last_launches = 0;
    cudaStream_t last_stream = nullptr;
    bool has_backward = false;
    unsigned long long* d_trace = nullptr;
    int trace_cap = 0;
    unsigned long long* d_cta_trace = nullptr;
    int cta_trace_phases = 0;
    int cta_trace_stride = 0;
    int last_grid = 0;
    int generation = 0;                          // bumped when the item workspace moves
    unsigned long long uid = 0;                  // unique over the process (never reused)
    // descriptors of the last batched combination led by this plan
    std::vector<unsigned long long> lzb_key;     // Lanczos batches: uids of the plans, in order
    std::vector<int> lzb_gens;
    rexi::LzArgs* d_lzb_args = nullptr;          // per-problem descriptors of the cached batch
    unsigned char* d_lzb_map = nullptr;          // problem of every CTA
    size_t lzb_cap_args = 0, lzb_cap_map = 0;
    int lzb_grid = 0;
    size_t lzb_smem = 0;
    std::vector<unsigned long long> batch_key;   // uids of the plans, in order
    std::vector<int> batch_gens;
    ProblemDesc* d_batch_prob = nullptr;
    ItemDesc* d_batch_items = nullptr;
    size_t batch_cap_prob = 0, batch_cap_items = 0;
    int batch_nitems = 0;
};

namespace {

int cuda_fail(cudaError_t e) { return e == cudaErrorMemoryAllocation ? REXI_ENOMEM : REXI_ECUDA; }

template <typename T>
int dalloc(rexi_plan* p, T** out, size_t count) {
    void* ptr = nullptr;
    cudaError_t e = cudaMalloc(&ptr, std::max<size_t>(count * sizeof(T), 16));
    if (e != cudaSuccess) { *out = nullptr; return cuda_fail(e); }
    p->allocs.push_back(ptr);
    *out = (T*)ptr;
    return REXI_OK;
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

bool finite_all(const double* v, size_t n) {
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(v[i])) return false;
    return true;
}

// diag_i = tau (V_i - c) - 2 sum_d a_d (the centred diagonal of tau H) in FP64 and FP32.
int upload_diag(rexi_plan* p, cudaStream_t stream, bool sync) {
    std::vector<double> d(p->n);
    std::vector<float> f(p->n);
    const double sa = 2.0 * (p->a[0] + p->a[1] + p->a[2]);
    for (int i = 0; i < p->n; ++i) {
        d[i] = p->tau * (p->V[i] - p->c) - sa;
        f[i] = (float)d[i];
    }
    cudaError_t e = cudaMemcpyAsync(p->d_diag, d.data(), sizeof(double) * p->n, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(p->d_diagf, f.data(), sizeof(float) * p->n, cudaMemcpyHostToDevice, stream);
    std::vector<double> dl;
    if (e == cudaSuccess && p->d_lz_diag) {
        // the Lanczos kernel's copy, divided by the stencil's fold factor
        dl.resize(p->n);
        for (int i = 0; i < p->n; ++i) dl[i] = d[i] / p->lz_fold;
        e = cudaMemcpyAsync(p->d_lz_diag, dl.data(), sizeof(double) * p->n, cudaMemcpyHostToDevice, stream);
    }
    std::vector<float2> dp;
    if (e == cudaSuccess && p->d_lz_diagdf && !dl.empty()) {
        // and as double-float pairs: hi = fl32(x), lo = fl32(x - hi)
        dp.resize(p->n);
        for (int i = 0; i < p->n; ++i) {
            const float hi = (float)dl[i];
            dp[i] = make_float2(hi, (float)(dl[i] - (double)hi));
        }
        e = cudaMemcpyAsync(p->d_lz_diagdf, dp.data(), sizeof(float2) * p->n, cudaMemcpyHostToDevice, stream);
    }
    // pageable host buffers: the copies have read them when the calls return;
    // sync waits for the device side as well
    if (e == cudaSuccess && sync) e = cudaStreamSynchronize(stream);
    return e == cudaSuccess ? REXI_OK : cuda_fail(e);
}

// Allocate the solver workspace for `nit` pole items (plus one group item per
// K poles when the first cycle is shared) and build descriptor sets.
int alloc_items(rexi_plan* p, int nit) {
    const size_t n = (size_t)p->n;
    const size_t esz = p->fp32 ? sizeof(float2) : sizeof(double2);
    const int ng = p->shared ? nit / p->K : 0;
    const int nall = nit + ng;
    int st;
    double2* x;
    void* basis;
    ItemState* sts;
    ItemStats* stats;
    double2 *p1, *p2;
    double* pn;
    if ((st = dalloc(p, &x, (size_t)nit * n))) return st;
    {
        void* ptr = nullptr;
        cudaError_t e = cudaMalloc(&ptr, (size_t)nall * (p->m + 1) * n * esz);
        if (e != cudaSuccess) return cuda_fail(e);
        p->allocs.push_back(ptr);
        basis = ptr;
    }
    if ((st = dalloc(p, &sts, (size_t)nall))) return st;
    if ((st = dalloc(p, &stats, (size_t)nall))) return st;
    if ((st = dalloc(p, &p1, (size_t)nall * p->max_tiles * p->pv))) return st;
    if ((st = dalloc(p, &p2, (size_t)nall * p->max_tiles * p->pv))) return st;
    if ((st = dalloc(p, &pn, (size_t)nall * p->max_tiles))) return st;
    if (ng > 0) {
        if ((st = dalloc(p, &p->d_gcs, (size_t)ng * rexi::kMaxM * p->K))) return st;
        if ((st = dalloc(p, &p->d_gsn, (size_t)ng * rexi::kMaxM * p->K))) return st;
    }
    p->ngroups = ng;
    p->d_x = x;
    p->d_basis = basis;
    p->d_st = sts;
    p->d_stats = stats;
    p->d_part1 = p1;
    p->d_part2 = p2;
    p->d_partn = pn;
    p->nit_cap = nit;
    p->generation++;
    return REXI_OK;
}

// Pole item in workspace slot idx; group_item is the launch-wide index of its
// shared-cycle group (-1: none).
ItemDesc make_item(const rexi_plan* p, int idx, int pole, bool adjoint, int problem, int group_item) {
    ItemDesc it{};
    it.problem = problem;
    it.pole = pole;
    it.adjoint = adjoint ? 1 : 0;
    it.tile_off = idx * p->max_tiles;            // offset inside this plan's partial buffers
    it.group = group_item;
    it.is_group = 0;
    it.tile = p->tile_pole;
    it.n = p->n;
    it.ntiles = (p->n + it.tile - 1) / it.tile;
    const cd s = p->z[pole] - p->tau * p->c;    // centred shift: A = tau (H - c) - s
    const cd sh = adjoint ? std::conj(s) : s;
    it.shift = make_double2(sh.real(), sh.imag());
    it.shiftf = make_float2((float)sh.real(), (float)sh.imag());
    const size_t esz = p->fp32 ? sizeof(float2) : sizeof(double2);
    if (idx >= p->nit_cap) return it;            // no item workspace (a Lanczos plan before its first adjoint)
    it.x = p->d_x + (size_t)idx * p->n;
    it.basis = (char*)p->d_basis + (size_t)idx * (p->m + 1) * p->n * esz;
    it.st = p->d_st + idx;
    it.stats = p->d_stats + idx;
    it.part1 = p->d_part1;
    it.part2 = p->d_part2;
    it.partn = p->d_partn;
    return it;
}

// Group item g (workspace slot nit_cap + g): Arnoldi on the unshifted operator
// tau (H - c) for members [member0, member0 + K) (launch-wide indices).
ItemDesc make_group(const rexi_plan* p, int g, bool adjoint, int problem, int member0) {
    ItemDesc it{};
    const int idx = p->nit_cap + g;
    it.problem = problem;
    it.pole = -1;
    it.adjoint = adjoint ? 1 : 0;
    it.tile_off = idx * p->max_tiles;
    it.n = p->n;
    it.tile = p->tile_group;
    it.ntiles = (p->n + it.tile - 1) / it.tile;
    it.shift = make_double2(0.0, 0.0);
    it.shiftf = make_float2(0.0f, 0.0f);
    it.x = nullptr;
    const size_t esz = p->fp32 ? sizeof(float2) : sizeof(double2);
    if (p->nit_cap == 0) return it;              // no item workspace
    it.basis = (char*)p->d_basis + (size_t)idx * (p->m + 1) * p->n * esz;
    it.group = -1;
    it.is_group = 1;
    it.member0 = member0;
    it.nmembers = p->K;
    it.gcs = p->d_gcs + (size_t)g * rexi::kMaxM * p->K;
    it.gsn = p->d_gsn + (size_t)g * rexi::kMaxM * p->K;
    it.st = p->d_st + idx;
    it.stats = p->d_stats + idx;
    it.part1 = p->d_part1;
    it.part2 = p->d_part2;
    it.partn = p->d_partn;
    return it;
}

// Items of one plan appended to a launch-wide list starting at `base`:
// poles first (the pole sum and the adjoint address them by pole index), then
// the group items.  backward: X poles, Y poles, X group, Y group.
void append_items(const rexi_plan* p, bool backward, int problem, int base, std::vector<ItemDesc>* out) {
    const int K = p->K;
    const int nsets = backward ? 2 : 1;
    for (int sset = 0; sset < nsets; ++sset)
        for (int k = 0; k < K; ++k) {
            const int grp = p->ngroups > 0 ? base + nsets * K + sset : -1;
            out->push_back(make_item(p, sset * K + k, k, sset == 1, problem, grp));
        }
    if (p->ngroups > 0)
        for (int sset = 0; sset < nsets; ++sset) out->push_back(make_group(p, sset, sset == 1, problem, base + sset * K));
}

ProblemDesc make_problem(const rexi_plan* p, int nsub, int item0, int nitems) {
    ProblemDesc pr{};
    pr.n = p->n;
    pr.nx = p->dims[0];
    pr.ny = p->dims[1];
    pr.nz = p->dims[2];
    pr.ntiles = p->ntiles;
    pr.K = p->K;
    pr.item0 = item0;
    pr.nitems = nitems;
    pr.nsub = nsub;
    for (int d = 0; d < 3; ++d) {
        pr.a[d] = p->a[d];
        pr.af[d] = (float)p->a[d];
    }
    pr.tau = p->tau;
    pr.alpha0 = make_double2(p->alpha0.real(), p->alpha0.imag());
    pr.alpha = p->d_alpha;
    pr.diag = p->d_diag;
    pr.diagf = p->d_diagf;
    pr.tmp0 = p->d_tmp0;
    pr.tmp1 = p->d_tmp1;
    pr.ckpt = p->d_ckpt;
    return pr;
}

int upload_set(rexi_plan* p, DescSet* set, const ProblemDesc& pr, const std::vector<ItemDesc>& items) {
    int st;
    if (!set->d_prob && (st = dalloc(p, &set->d_prob, 1))) return st;
    if (set->nitems < (int)items.size() || !set->d_items) {
        if ((st = dalloc(p, &set->d_items, items.size()))) return st;
    }
    set->nitems = (int)items.size();
    set->ntiles_items = 0;
    for (const ItemDesc& it : items) set->ntiles_items += it.ntiles;
    cudaError_t e = cudaMemcpy(set->d_prob, &pr, sizeof(pr), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(set->d_items, items.data(), sizeof(ItemDesc) * items.size(), cudaMemcpyHostToDevice);
    return e == cudaSuccess ? REXI_OK : cuda_fail(e);
}

int build_sets(rexi_plan* p) {
    std::vector<ItemDesc> f;
    append_items(p, false, 0, 0, &f);
    p->hprob = make_problem(p, p->n_sub, 0, (int)f.size());
    int st = upload_set(p, &p->fwd, p->hprob, f);
    if (st) return st;
    st = upload_set(p, &p->one, make_problem(p, 1, 0, (int)f.size()), f);
    if (st) return st;
    if (p->nit_cap >= 2 * p->K) {
        std::vector<ItemDesc> b;
        append_items(p, true, 0, 0, &b);
        st = upload_set(p, &p->bwd, make_problem(p, p->n_sub, 0, (int)b.size()), b);
        if (st) return st;
        p->has_backward = true;
    }
    return REXI_OK;
}

int ensure_backward(rexi_plan* p) {
    if (p->has_backward) return REXI_OK;
    // re-allocate the item workspace for 2K items and the substep checkpoints
    int st = alloc_items(p, 2 * p->K);
    if (st) return st;
    if ((st = dalloc(p, &p->d_ckpt, (size_t)std::max(1, p->n_sub) * p->n))) return st;
    return build_sets(p);
}

EngineArgs base_args(const rexi_plan* p, int mode, const DescSet& set, int nproblems, int max_sub) {
    EngineArgs A{};
    A.mode = mode;
    A.nproblems = nproblems;
    A.nitems = set.nitems;
    A.m = p->m;
    A.max_iters = p->opt.max_iters;
    A.max_sub = max_sub;
    A.pv = p->pv;
    A.ortho = p->eng_ortho;
    A.window = p->eng_window;
    A.tol = p->tol;
    A.inner_tol = p->fp32 ? p->opt.inner_tol : 0.0;
    A.timeout_ns = p->timeout_ns;
    A.prob = set.d_prob;
    A.item = set.d_items;
    A.bar = p->d_bar;
    A.epoch = p->d_bar + 2;
    A.err = p->d_err;
    A.bytes = p->d_bytes;
    A.trace = p->trace_cap > 0 ? p->d_trace : nullptr;
    A.trace_cap = p->trace_cap;
    A.cta_trace = p->cta_trace_phases > 0 ? p->d_cta_trace : nullptr;
    A.cta_trace_phases = p->cta_trace_phases;
    A.cta_trace_stride = p->cta_trace_stride;
    return A;
}

// Largest co-resident grid of the persistent kernel (cooperative launch limit).
int max_grid_cached(bool fp32, size_t smem, int device, bool wide) {
    static std::mutex mu;
    static std::vector<std::pair<std::pair<int, size_t>, int>> cache;
    const std::pair<int, size_t> key(device * 4 + (fp32 ? 1 : 0) + (wide ? 2 : 0), smem);
    {
        std::lock_guard<std::mutex> lk(mu);
        for (auto& c : cache)
            if (c.first == key) return c.second;
    }
    const int g = rexi::engine_max_grid(fp32, smem, device, wide);
    if (g > 0) {
        std::lock_guard<std::mutex> lk(mu);
        cache.push_back(std::make_pair(key, g));
    }
    return g;
}

int sm_count(int device) {
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return 1;
    return std::max(1, sms);
}

int launch(rexi_plan* p, const EngineArgs& A, const IOArgs& io, int total_tiles, cudaStream_t stream) {
    cudaError_t e = cudaMemsetAsync(p->d_bar, 0, 3 * sizeof(unsigned), stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->d_err, 0, sizeof(int), stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->d_bytes, 0, 3 * sizeof(unsigned long long), stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->d_stats, 0, sizeof(ItemStats) * A.nitems, stream);
    if (e != cudaSuccess) return cuda_fail(e);
    const size_t smem = rexi::engine_smem_bytes(A.nitems, p->fp32, A.ortho);
    const bool wide = !p->fp32 && p->ctas_per_sm == 1;     // one CTA per SM: the wide-register kernel
    int maxg = max_grid_cached(p->fp32, smem, p->device, wide);
    if (maxg <= 0) return REXI_ECUDA;
    if (p->ctas_per_sm > 0) maxg = std::min(maxg, p->ctas_per_sm * sm_count(p->device));
    const int grid = std::max(1, std::min(maxg, total_tiles));
    e = rexi::launch_engine(p->fp32, A, io, grid, smem, stream, wide);
    p->last_stream = stream;
    p->last_launches = 1;
    p->last_grid = grid;
    return e == cudaSuccess ? REXI_OK : cuda_fail(e);
}

// Read back the error word and the per-item statistics (synchronises).
int collect(rexi_plan* p, cudaStream_t stream, int nitems, int item_offset, int poles, rexi_stats* st,
            int n_sub) {
    int err = 0;
    unsigned long long nbytes[3] = {0, 0, 0};
    std::vector<ItemStats> s(nitems);
    cudaError_t e = cudaMemcpyAsync(&err, p->d_err, sizeof(int), cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(nbytes, p->d_bytes, sizeof(nbytes), cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(s.data(), p->d_stats, sizeof(ItemStats) * nitems, cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return cuda_fail(e);
    int status = err != 0 ? err : REXI_OK;
    bool failed = false;
    for (const ItemStats& x : s) failed = failed || x.failed;
    if (status == REXI_OK && failed) status = REXI_ENOCONV;
    if (st) {
        std::memset(st, 0, sizeof(*st));
        st->n_sub = n_sub;
        for (int k = 0; k < poles && k < REXI_MAX_POLES; ++k) {
            const ItemStats& x = s[item_offset + k];
            st->iters[k] = x.iters;
            st->cycles[k] = x.cycles;
            st->iters_sq[k] = x.iters_sq;
            st->resid[k] = x.resid;
        }
        for (const ItemStats& x : s) {
            st->total_iters += x.iters;
            st->total_cycles += x.cycles;
            st->max_iters_seen = std::max(st->max_iters_seen, x.max_sub_iters);
        }
        st->status = status;
        st->bytes = (double)nbytes[0];
        st->flops64 = (double)nbytes[1];
        st->ops32 = (double)nbytes[2];
    }
    return status;
}

// ---- shared-basis Lanczos path ----------------------------------------------

// Tile box of the Lanczos kernel: the box (at most `target` interior points,
// tile plus halo within the kernel's staging limit, shared memory for the
// requested CTAs per SM) that minimises the work of the busiest SM, counting
// 10 units per interior point (update and stencil), 6 per point of the
// extended box (the update, recomputed on the halo) and 4600 per tile, with tile t on CTA
// 1 + t mod (G - 1) and CTA c on SM c mod (SMs) (the order in which the
// resident grid fills the SMs).  Then the grid, the dynamic shared memory and
// the rows the control CTA stages per chunk.
// Tile box and shared memory of one problem run by G CTAs (one control CTA
// and G - 1 tile CTAs) at cps CTAs per SM; the load model spreads the tile
// CTAs over model_sms SMs.
struct LzChoice {
    int tx = 1, ty = 1, tz = 1;
    bool resident = false;
    size_t smem = 0;
    int stage = 1;
};

int lz_choose(const rexi_plan* p, int G, int cps, int model_sms, LzChoice* out) {
    const int sms = std::max(1, model_sms);
    const int hx = p->a[0] != 0.0 ? 1 : 0, hy = p->a[1] != 0.0 ? 1 : 0, hz = p->a[2] != 0.0 ? 1 : 0;
    const int nx = p->dims[0], ny = p->dims[1], nz = p->dims[2];
    const int target = p->lz_target > 0 ? std::min(p->lz_target, rexi::kLzMaxInterior) : rexi::kLzMaxInterior;
    const int tile_ctas = std::max(1, G - 1);
    int smem_sm = 0;
    if (cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, p->device) != cudaSuccess)
        return REXI_ECUDA;
    const size_t stat = rexi::lanczos_static_smem();
    const size_t per_cta = (size_t)smem_sm / cps;
    const size_t row_bytes = (size_t)p->K * 3 * sizeof(double2);
    const size_t ctl_min = std::min<size_t>(8 * row_bytes, 96 * 1024);
    long long best = -1;
    int bx = 1, by = 1, bz = 1;
    const int widths[] = {16, 32, 64, 128, 256, 512, 1024, 2048};
    std::vector<int> txs;
    for (int w : widths)
        if (w < nx) txs.push_back(w);
    if (nx <= 2048) txs.push_back(nx);
    std::vector<long long> load(sms);
    for (int tx : txs) {
        if (tx > target) continue;
        for (int tz = 1; tz <= std::min(nz, target / tx); ++tz) {
            for (int ty = 1; ty <= std::min(ny, target / (tx * tz)); ++ty) {
                const long long E = (long long)(tx + 2 * hx) * (ty + 2 * hy) * (tz + 2 * hz);
                if (E > rexi::kLzMaxExt) continue;
                const size_t smem = std::max(rexi::lanczos_smem_bytes(tx, ty, tz, hx, hy, hz, false), ctl_min);
                if (smem + stat + 1024 > per_cta) continue;
                const int gx = (nx + tx - 1) / tx, gy = (ny + ty - 1) / ty, gz = (nz + tz - 1) / tz;
                const long long ntiles = (long long)gx * gy * gz;
                if (ntiles > 64LL * tile_ctas) continue;
                std::fill(load.begin(), load.end(), 0LL);
                long long worst = 0;
                for (long long t = 0; t < ntiles; ++t) {
                    // the actual (ragged) extent of tile t
                    const int ix = (int)(t % gx), iy = (int)((t / gx) % gy), iz = (int)(t / ((long long)gx * gy));
                    const long long ax = std::min(tx, nx - ix * tx), ay = std::min(ty, ny - iy * ty),
                                    az = std::min(tz, nz - iz * tz);
                    // plus a fixed cost per tile (staging, three CTA barriers), measured
                    // at about the work of 450 interior points
                    const long long cost =
                        10 * ax * ay * az + 6 * (ax + 2 * hx) * (ay + 2 * hy) * (az + 2 * hz) + 4600;
                    const int sm_of = (int)((1 + t % tile_ctas) % sms);
                    load[sm_of] += cost;
                    worst = std::max(worst, load[sm_of]);
                }
                if (best < 0 || worst < best || (worst == best && tx > bx)) {
                    best = worst;
                    bx = tx;
                    by = ty;
                    bz = tz;
                }
            }
        }
    }
    if (best < 0) return REXI_EINVAL;               // no box fits (a row longer than 2048 points)
    out->tx = bx;
    out->ty = by;
    out->tz = bz;
    // resident mode when every tile CTA owns at most one tile and its state fits
    const long long ntiles = (long long)((nx + bx - 1) / bx) * ((ny + by - 1) / by) * ((nz + bz - 1) / bz);
    const size_t smem_res = std::max(rexi::lanczos_smem_bytes(bx, by, bz, hx, hy, hz, true), ctl_min);
    out->resident = ntiles <= tile_ctas && smem_res + stat + 1024 <= per_cta;
    out->smem =
        out->resident ? smem_res : std::max(rexi::lanczos_smem_bytes(bx, by, bz, hx, hy, hz, false), ctl_min);
    out->stage = (int)std::max<size_t>(1, std::min<size_t>(64, out->smem / row_bytes));
    return REXI_OK;
}

int lz_configure(rexi_plan* p) {
    const int sms = sm_count(p->device);
    const int cps = std::max(1, std::min(p->lz_cps, 8));
    const int G = cps * sms;
    LzChoice c;
    const int r = lz_choose(p, G, cps, sms, &c);
    if (r) return r;
    p->lz_tx = c.tx;
    p->lz_ty = c.ty;
    p->lz_tz = c.tz;
    p->lz_resident = c.resident;
    p->lz_stage = c.stage;
    p->lz_smem = c.smem;
    const size_t smem = c.smem;
    const int maxg = rexi::lanczos_max_grid(smem, p->device);
    if (maxg < 2) return REXI_ECUDA;
    p->lz_grid = std::min(maxg, G);
    if (p->lz_grid > p->lz_part_cap) return REXI_EINVAL;
    return REXI_OK;
}

int lz_alloc(rexi_plan* p) {
    const size_t n = (size_t)p->n, K = (size_t)p->K, m = (size_t)p->lz_m;
    int st;
    p->lz_part_cap = 8 * sm_count(p->device);
    if ((st = dalloc(p, &p->d_lz_basis, (m + 2) * n))) return st;
    if ((st = dalloc(p, &p->d_lz_wt, 2 * n))) return st;
    if ((st = dalloc(p, &p->d_lz_part, 2 * (size_t)p->lz_part_cap))) return st;
    if ((st = dalloc(p, &p->d_lz_rows, m * K * 3))) return st;
    if ((st = dalloc(p, &p->d_lz_ybuf, m * K))) return st;
    if ((st = dalloc(p, &p->d_lz_coef, m * K))) return st;
    if ((st = dalloc(p, &p->d_lz_rho, m + 2))) return st;
    if ((st = dalloc(p, &p->d_lz_stop, (size_t)std::max(1, p->n_sub)))) return st;
    if ((st = dalloc(p, &p->d_lz_cols, 2 * (size_t)std::max(1, p->n_sub)))) return st;
    if ((st = dalloc(p, &p->d_lz_shift, K))) return st;
    // f = |first nonzero stencil coefficient| (the coefficients are negative)
    p->lz_fold = std::fabs(p->a[0] != 0.0 ? p->a[0] : (p->a[1] != 0.0 ? p->a[1] : (p->a[2] != 0.0 ? p->a[2] : 1.0)));
    if ((st = dalloc(p, &p->d_lz_diag, n))) return st;
    if ((st = dalloc(p, &p->d_lz_diagdf, n))) return st;
    if ((st = upload_diag(p, 0, true))) return st;
#ifdef REXI_DEBUG
    if ((st = dalloc(p, &p->d_dbg, 4))) return st;
    if (cudaMemset(p->d_dbg, 0, 4 * sizeof(long long)) != cudaSuccess) return REXI_ECUDA;
#endif
    if (!p->d_stats && (st = dalloc(p, &p->d_stats, K))) return st;
    std::vector<double2> sh(K);
    for (size_t k = 0; k < K; ++k) {
        const cd v = p->z[k] - p->tau * p->c;
        sh[k] = make_double2(v.real(), v.imag());
    }
    if (cudaMemcpy(p->d_lz_shift, sh.data(), sizeof(double2) * K, cudaMemcpyHostToDevice) != cudaSuccess)
        return REXI_ECUDA;
    return lz_configure(p);
}

// One launch of the Lanczos kernel: n_sub substeps (mode LZ_STEP) or the K
// solves of one substep (LZ_SOLVE, x = out [K][n]).
rexi::LzArgs lz_args(rexi_plan* p, int mode, const void* in, void* out, const LzChoice& c, int cta0, int ncta);

int lz_launch(rexi_plan* p, int mode, const void* in, void* out, cudaStream_t stream) {
    const int nsub = mode == rexi::LZ_STEP ? p->n_sub : 1;
    cudaError_t e = cudaMemsetAsync(p->d_bar, 0, 3 * sizeof(unsigned), stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->d_err, 0, sizeof(int), stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->d_bytes, 0, 3 * sizeof(unsigned long long), stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->d_stats, 0, sizeof(ItemStats) * p->K, stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->d_lz_stop, 0xFF, sizeof(int) * nsub, stream);
    if (e == cudaSuccess && p->d_dbg) e = cudaMemsetAsync(p->d_dbg, 0, 4 * sizeof(long long), stream);
    if (e != cudaSuccess) return cuda_fail(e);
    LzChoice c;
    c.tx = p->lz_tx;
    c.ty = p->lz_ty;
    c.tz = p->lz_tz;
    c.resident = p->lz_resident;
    c.stage = p->lz_stage;
    const rexi::LzArgs A = lz_args(p, mode, in, out, c, 0, p->lz_grid);
    e = rexi::launch_lanczos(A, p->lz_grid, p->lz_smem, stream);
    p->last_stream = stream;
    p->last_launches = 1;
    p->last_grid = p->lz_grid;
    return e == cudaSuccess ? REXI_OK : cuda_fail(e);
}

// The descriptor of one Lanczos launch of plan p (tile choice c, CTAs cta0 ..
// cta0 + ncta - 1 of the launch).
rexi::LzArgs lz_args(rexi_plan* p, int mode, const void* in, void* out, const LzChoice& c, int cta0, int ncta) {
    const int nsub = mode == rexi::LZ_STEP ? p->n_sub : 1;
    rexi::LzArgs A{};
    A.mode = mode;
    A.n = p->n;
    A.nx = p->dims[0];
    A.ny = p->dims[1];
    A.nz = p->dims[2];
    A.K = p->K;
    A.nsub = nsub;
    A.m = std::min(p->lz_m, p->opt.max_iters);
    for (int d = 0; d < 3; ++d) {
        A.a[d] = p->a[d];
        A.ratio[d] = p->a[d] / p->lz_fold;
    }
    A.fold = p->lz_fold;
    // the unscaled recurrence grows a vector by at most ||B|| / f = tau W / f
    // per step; below 2^16 its norms stay far inside the FP32 range of the
    // compensated inner products between rescalings
    A.unit_ok = p->tau * p->W / p->lz_fold <= 65536.0 ? 1 : 0;
    A.diag = p->d_lz_diag;
    A.diag_df = p->d_lz_diagdf;
    A.df = p->opt.precision == REXI_DF64 ? 1 : 0;
    A.shift = p->d_lz_shift;
    A.alpha = p->d_alpha;
    A.alpha0 = make_double2(p->alpha0.real(), p->alpha0.imag());
    A.tol = p->tol;
    A.stage_rows = c.stage;
    A.tx = c.tx;
    A.ty = c.ty;
    A.tz = c.tz;
    A.gx = (A.nx + A.tx - 1) / A.tx;
    A.gy = (A.ny + A.ty - 1) / A.ty;
    A.gz = (A.nz + A.tz - 1) / A.tz;
    A.ntiles = A.gx * A.gy * A.gz;
    A.resident = c.resident ? 1 : 0;
    A.in = (const double2*)in;
    A.out = (double2*)out;
    A.tmp0 = p->d_tmp0;
    A.tmp1 = p->d_tmp1;
    A.basis = p->d_lz_basis;
    A.wt = p->d_lz_wt;
    A.part = p->d_lz_part;
    A.rows = p->d_lz_rows;
    A.ybuf = p->d_lz_ybuf;
    A.coef = p->d_lz_coef;
    A.rho = p->d_lz_rho;
    A.stop = p->d_lz_stop;
    A.cols = p->d_lz_cols;
    A.stats = p->d_stats;
    A.bar = p->d_bar;
    A.err = p->d_err;
    A.timeout_ns = p->timeout_ns;
    A.trace = p->trace_cap > 0 ? p->d_trace : nullptr;
    A.trace_cap = p->trace_cap;
    A.bytes = p->d_bytes;
    A.part_cap = p->lz_part_cap;
    A.dbg = p->d_dbg;
    A.dbg_trip = p->dbg_trip;
    A.cta0 = cta0;
    A.ncta = ncta;
    return A;
}

// One step of several problems in one launch of the Lanczos kernel: the CTAs
// are divided among the problems in proportion to their work (each problem
// gets a control CTA and at least one tile CTA), every problem's tile boxes are
// chosen for its share, and every problem synchronises only its own CTAs.
// The descriptors are cached in the first plan, keyed like the item engine's.
int lz_step_batched(rexi_plan* const* plans, int B, const void* const* psi_in, void* const* psi_out, cudaStream_t s,
                    rexi_stats* st) {
    rexi_plan* p0 = plans[0];
    const int sms = sm_count(p0->device);
    const int cps = 2;
    std::vector<unsigned long long> key(B);
    std::vector<int> gens(B);
    for (int b = 0; b < B; ++b) {
        key[b] = plans[b]->uid;
        gens[b] = plans[b]->generation;
    }
    if (p0->lzb_key != key || p0->lzb_gens != gens || !p0->d_lzb_args) {
        int G = cps * sms;
        if (G < 2 * B) return REXI_EINVAL;                  // a control and a tile CTA per problem
        // CTAs in proportion to the work (points x substeps), at least two per problem
        long long N = 0;
        for (int b = 0; b < B; ++b) N += (long long)plans[b]->n * plans[b]->n_sub;
        std::vector<int> nct(B);
        int used = 0;
        for (int b = 0; b < B; ++b) {
            nct[b] = 2 + (int)((long long)(G - 2 * B) * plans[b]->n * plans[b]->n_sub / N);
            used += nct[b];
        }
        for (int b = 0; used < G; b = (b + 1) % B, ++used) ++nct[b];
        std::vector<LzChoice> ch(B);
        size_t smem = 0;
        for (int b = 0; b < B; ++b) {
            const int r = lz_choose(plans[b], nct[b], cps, nct[b], &ch[b]);
            if (r) return r;
            smem = std::max(smem, ch[b].smem);
        }
        const int maxg = rexi::lanczos_max_grid(smem, p0->device, true);
        if (maxg < G) return REXI_ECUDA;
        std::vector<rexi::LzArgs> args(B);
        std::vector<unsigned char> map(G);
        int c0 = 0;
        for (int b = 0; b < B; ++b) {
            rexi_plan* p = plans[b];
            if (nct[b] > p->lz_part_cap) return REXI_EINVAL;
            // the control CTA stages rows in the launch's dynamic shared memory
            ch[b].stage = (int)std::max<size_t>(1, std::min<size_t>(64, smem / ((size_t)p->K * 3 * sizeof(double2))));
            args[b] = lz_args(p, rexi::LZ_STEP, nullptr, nullptr, ch[b], c0, nct[b]);
            args[b].trace = nullptr;
            args[b].trace_cap = 0;
            for (int c = 0; c < nct[b]; ++c) map[c0 + c] = (unsigned char)b;
            c0 += nct[b];
        }
        if (cudaStreamSynchronize(s) != cudaSuccess) return REXI_ECUDA;   // old descriptors may be in use
        int r;
        if ((size_t)B > p0->lzb_cap_args) {
            if ((r = dalloc(p0, &p0->d_lzb_args, (size_t)B))) return r;
            p0->lzb_cap_args = (size_t)B;
        }
        if ((size_t)G > p0->lzb_cap_map) {
            if ((r = dalloc(p0, &p0->d_lzb_map, (size_t)G))) return r;
            p0->lzb_cap_map = (size_t)G;
        }
        p0->lzb_key.clear();                     // invalid until the copies succeed
        if (cudaMemcpy(p0->d_lzb_args, args.data(), sizeof(rexi::LzArgs) * B, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(p0->d_lzb_map, map.data(), (size_t)G, cudaMemcpyHostToDevice) != cudaSuccess)
            return REXI_ECUDA;
        p0->lzb_key = key;
        p0->lzb_gens = gens;
        p0->lzb_grid = G;
        p0->lzb_smem = smem;
    }
    rexi::LzIO io{};
    for (int b = 0; b < B; ++b) {
        io.in[b] = (const double2*)psi_in[b];
        io.out[b] = (double2*)psi_out[b];
    }
    cudaError_t e = rexi::lanczos_reset(p0->d_lzb_args, B, s);
    if (e == cudaSuccess)
        e = rexi::launch_lanczos_batched(p0->d_lzb_args, p0->d_lzb_map, io, p0->lzb_grid, p0->lzb_smem, s);
    for (int b = 0; b < B; ++b) {
        plans[b]->last_stream = s;
        plans[b]->last_launches = 1;
        plans[b]->last_grid = p0->lzb_grid;
    }
    if (e != cudaSuccess) return cuda_fail(e);
    if (!st) return REXI_OK;
    int status = REXI_OK;
    for (int b = 0; b < B; ++b) {
        const int r = collect(plans[b], s, plans[b]->K, 0, plans[b]->K, &st[b], plans[b]->n_sub);
        plans[b]->last_status = r;
        if (r != REXI_OK && status == REXI_OK) status = r;
    }
    return status;
}

}  // namespace

extern "C" {

const char* rexi_status_string(int s) {
    switch (s) {
        case REXI_OK: return "REXI_OK";
        case REXI_EINVAL: return "REXI_EINVAL: invalid argument";
        case REXI_ENOMEM: return "REXI_ENOMEM: allocation failed";
        case REXI_ECUDA: return "REXI_ECUDA: CUDA runtime error";
        case REXI_ENOCONV: return "REXI_ENOCONV: a pole solve did not converge";
        case REXI_ETIMEOUT: return "REXI_ETIMEOUT: bounded device wait expired";
        case REXI_EPLAN: return "REXI_EPLAN: FCF construction failed";
        case REXI_EBOUNDS: return "REXI_EBOUNDS: an index check of the debug build failed (access skipped)";
        case REXI_WACCURACY: return "REXI_WACCURACY: accuracy condition (Eq. (10)) violated";
        default: return "unknown status";
    }
}

int rexi_options_default(rexi_options* o) {
    if (!o) return REXI_EINVAL;
    std::memset(o, 0, sizeof(*o));
    o->precision = REXI_MIXED;
    o->restart_m = 30;
    o->max_iters = 2000;
    o->tol = 0.0;
    o->inner_tol = 1e-5;
    o->R1 = 0.0;
    o->eps_target = 1e-9;
    o->allow_substeps = 1;
    o->stabilize_eps = 0.0;
    o->want_backward = 0;
    o->device = -1;
    o->shared_first_cycle = 1;
    o->ortho = 1;
    o->window = 0;
    return REXI_OK;
}

int rexi_fcf(int K, double R1, double eps_target, double* sigma, double* beta, double* R1_used,
             double* sigma_K1, double* min_re_sigma, double* amplification) {
    if (K < 1 || K > REXI_MAX_POLES || !(R1 >= 0.0) || !std::isfinite(R1)) return REXI_EINVAL;
    if (!(eps_target > 0.0)) eps_target = 1e-9;
    const double R = R1 > 0.0 ? R1 : rexi::fcf_default_R1_cached(K, eps_target);
    rexi::FcfResult r;
    const int st = rexi::fcf_cached(K, R, &r);
    if (R1_used) *R1_used = R;
    if (st != 0) return st == -1 ? REXI_EINVAL : REXI_EPLAN;
    for (int k = 0; k < K; ++k) {
        if (sigma) { sigma[2 * k] = r.sigma[k].real(); sigma[2 * k + 1] = r.sigma[k].imag(); }
        if (beta) { beta[2 * k] = r.beta[k].real(); beta[2 * k + 1] = r.beta[k].imag(); }
    }
    if (sigma_K1) *sigma_K1 = r.sigma_K1;
    if (min_re_sigma) *min_re_sigma = r.min_re_sigma;
    if (amplification) *amplification = r.amplification;
    return REXI_OK;
}

int rexi_plan_create(rexi_plan** out, const rexi_grid* g, const double* V, double dt, int K,
                     const rexi_options* opt_in) {
    if (!out) return REXI_EINVAL;
    *out = nullptr;
    if (!g || !V || !(dt > 0.0) || !std::isfinite(dt) || K < 1 || K > REXI_MAX_POLES) return REXI_EINVAL;
    if (g->ndim < 1 || g->ndim > 3 || !(g->hbar > 0.0) || !(g->mass > 0.0)) return REXI_EINVAL;
    rexi_options opt;
    if (opt_in) opt = *opt_in; else rexi_options_default(&opt);
    if (opt.precision != REXI_FP64 && opt.precision != REXI_MIXED && opt.precision != REXI_DF64) return REXI_EINVAL;
    if (opt.restart_m < 1 || opt.max_iters < 1) return REXI_EINVAL;
    if (opt.ortho < 0 || opt.ortho > 2) return REXI_EINVAL;
    const bool lanczos = opt.ortho == 2;
    if (lanczos) {
        // one shared basis per substep, no restarts: FP64 or double-float, no window
        if (opt.precision == REXI_MIXED || opt.window != 0 || opt.restart_m > REXI_MAX_KRYLOV) return REXI_EINVAL;
    } else {
        if (opt.precision == REXI_DF64) return REXI_EINVAL;   // the double-float form is the Lanczos kernel's
        if (opt.restart_m > REXI_MAX_RESTART) return REXI_EINVAL;
        // full orthogonalisation keeps m + 1 dot products per step in registers
        if (opt.window == 0 &&
            opt.restart_m > (opt.ortho == 1 ? REXI_MAX_RESTART_FULL : REXI_MAX_RESTART_FULL + 1))
            return REXI_EINVAL;
        if (opt.window < 0 || opt.window == 1 || opt.window > REXI_MAX_RESTART || (opt.window > 0 && opt.ortho != 1))
            return REXI_EINVAL;
    }
    if (!(opt.tol >= 0.0) || !(opt.R1 >= 0.0) || !(opt.inner_tol >= 0.0) || !(opt.stabilize_eps >= 0.0) ||
        !(opt.stabilize_eps < 1.0))
        return REXI_EINVAL;
    long long n = 1;
    int dims[3] = {1, 1, 1};
    double h[3] = {1.0, 1.0, 1.0};
    for (int d = 0; d < g->ndim; ++d) {
        if (g->n[d] < 1 || !(g->hi[d] > g->lo[d]) || !std::isfinite(g->hi[d] - g->lo[d])) return REXI_EINVAL;
        if (n > (1ll << 30) / g->n[d]) return REXI_EINVAL;   // checked before the product can overflow
        dims[d] = g->n[d];
        h[d] = (g->hi[d] - g->lo[d]) / g->n[d];
        n *= g->n[d];
    }
    if (!finite_all(V, (size_t)n)) return REXI_EINVAL;

    static std::atomic<unsigned long long> next_uid{1};
    rexi_plan* p = new (std::nothrow) rexi_plan();
    if (!p) return REXI_ENOMEM;
    p->uid = next_uid.fetch_add(1);
    p->grid = *g;
    p->opt = opt;
    p->n = (int)n;
    p->K = K;
    p->m = opt.restart_m;
    p->eng_ortho = opt.ortho;
    p->eng_window = opt.window;
    if (lanczos) {
        // the item engine serves the adjoint of a Lanczos plan: shared first
        // cycle, two-vector window, restart length up to 64
        p->lanczos = true;
        p->lz_m = opt.restart_m;
        p->m = std::min(opt.restart_m, REXI_MAX_RESTART);
        p->eng_ortho = 1;
        p->eng_window = 2;
    }
    p->dt = dt;
    p->fp32 = opt.precision == REXI_MIXED;
    p->shared = opt.shared_first_cycle != 0;
    for (int d = 0; d < 3; ++d) { p->dims[d] = dims[d]; p->h[d] = h[d]; }
    p->V.assign(V, V + n);

    // spectral enclosure of H (exact bound of the periodic Laplacian plus diag(V))
    double vmin = V[0], vmax = V[0];
    for (long long i = 1; i < n; ++i) { vmin = std::min(vmin, V[i]); vmax = std::max(vmax, V[i]); }
    double kin = 0.0;
    for (int d = 0; d < g->ndim; ++d) kin += 4.0 / (h[d] * h[d]);
    kin *= g->hbar * g->hbar / (2.0 * g->mass);
    p->E_min = vmin;
    p->E_max = vmax + kin;
    p->c = 0.5 * (p->E_min + p->E_max);
    p->W = 0.5 * (p->E_max - p->E_min);

    // R1, FCF poles and weights (Algorithms 1-2), substeps (Eq. (10))
    const double eps_t = opt.eps_target > 0.0 ? opt.eps_target : 1e-9;
    p->R1 = opt.R1 > 0.0 ? opt.R1 : rexi::fcf_default_R1_cached(K, eps_t);
    int fst = rexi::fcf_cached(K, p->R1, &p->fcf);
    if (fst != 0) { delete p; return fst == -1 ? REXI_EINVAL : REXI_EPLAN; }
    const double x = dt * p->W / (g->hbar * p->R1);
    if (opt.allow_substeps) {
        p->n_sub = std::max(1, (int)std::ceil(x - 1e-12 * std::max(1.0, x)));
    } else {
        p->n_sub = 1;
        if (x > 1.0 + 1e-12) p->warn = REXI_WACCURACY;
    }
    p->tau = dt / p->n_sub;
    p->z.resize(K);
    p->alpha.resize(K);
    const cd I(0.0, 1.0);
    const cd phase = std::exp(-I * (p->tau * p->c / g->hbar));
    for (int k = 0; k < K; ++k) {
        const cd beta = p->fcf.beta[k] * (1.0 - opt.stabilize_eps);
        p->z[k] = p->tau * p->c + I * g->hbar * p->fcf.sigma[k];
        p->alpha[k] = I * g->hbar * beta * phase;
    }
    p->alpha0 = 0.0;
    // A dimension of length 1 contributes (u + u - 2u)/h^2 = 0 to the periodic Laplacian: drop it.
    for (int d = 0; d < g->ndim; ++d)
        p->a[d] = dims[d] > 1 ? -p->tau * g->hbar * g->hbar / (2.0 * g->mass * h[d] * h[d]) : 0.0;
    p->tol = opt.tol > 0.0 ? opt.tol
                           : std::max(2e-14, std::min(1e-10, 1e-6 / std::max(1.0, p->fcf.amplification)));
    p->ntiles = (p->n + rexi::kTile - 1) / rexi::kTile;
    p->max_tiles = (p->n + rexi::kBlock - 1) / rexi::kBlock;
    p->pv = 40;

    // device
    int dev = opt.device;
    if (dev < 0 && cudaGetDevice(&dev) != cudaSuccess) { delete p; return REXI_ECUDA; }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || dev >= ndev) { delete p; return REXI_ECUDA; }
    p->device = dev;
    DeviceGuard guard(dev);
    int st;
    auto fail = [&](int code) { rexi_plan_destroy(p); return code; };
    if ((st = dalloc(p, &p->d_diag, n))) return fail(st);
    if ((st = dalloc(p, &p->d_diagf, n))) return fail(st);
    if ((st = dalloc(p, &p->d_alpha, K))) return fail(st);
    if ((st = dalloc(p, &p->d_tmp0, n))) return fail(st);
    if ((st = dalloc(p, &p->d_tmp1, n))) return fail(st);
    if ((st = dalloc(p, &p->d_hin, n))) return fail(st);
    if ((st = dalloc(p, &p->d_hout, n))) return fail(st);
    if ((st = dalloc(p, &p->d_bar, 4))) return fail(st);
    if ((st = dalloc(p, &p->d_err, 1))) return fail(st);
    if ((st = dalloc(p, &p->d_bytes, 3))) return fail(st);
    {
        std::vector<double2> al(K);
        for (int k = 0; k < K; ++k) al[k] = make_double2(p->alpha[k].real(), p->alpha[k].imag());
        if (cudaMemcpy(p->d_alpha, al.data(), sizeof(double2) * K, cudaMemcpyHostToDevice) != cudaSuccess)
            return fail(REXI_ECUDA);
    }
    if ((st = upload_diag(p, 0, true))) return fail(st);
    if (cudaMemset(p->d_bar, 0, 4 * sizeof(unsigned)) != cudaSuccess) return fail(REXI_ECUDA);
    if (cudaMemset(p->d_err, 0, sizeof(int)) != cudaSuccess) return fail(REXI_ECUDA);
    if (opt.want_backward) {
        if ((st = alloc_items(p, 2 * K))) return fail(st);
        if ((st = dalloc(p, &p->d_ckpt, (size_t)std::max(1, p->n_sub) * n))) return fail(st);
    } else if (!p->lanczos) {
        if ((st = alloc_items(p, K))) return fail(st);
    }
    if (p->lanczos && (st = lz_alloc(p))) return fail(st);
    if ((st = build_sets(p))) return fail(st);
    *out = p;
    return p->warn;
}

void rexi_plan_destroy(rexi_plan* p) {
    if (!p) return;
    DeviceGuard guard(p->device);
    for (void* a : p->allocs) cudaFree(a);
    delete p;
}

int rexi_plan_get_info(const rexi_plan* p, rexi_plan_info* info) {
    if (!p || !info) return REXI_EINVAL;
    std::memset(info, 0, sizeof(*info));
    info->K = p->K;
    info->n_sub = p->n_sub;
    info->n_total = p->n;
    info->restart_m = p->lanczos ? p->lz_m : p->m;
    info->precision = p->opt.precision;
    info->dt = p->dt;
    info->tau = p->tau;
    info->R1 = p->R1;
    info->sigma_K1 = p->fcf.sigma_K1;
    info->E_min = p->E_min;
    info->E_max = p->E_max;
    info->c = p->c;
    info->W = p->W;
    info->amplification = p->fcf.amplification;
    info->tol = p->tol;
    info->min_re_sigma = p->fcf.min_re_sigma;
    return REXI_OK;
}

int rexi_plan_poles(const rexi_plan* p, double* z, double* alpha, double* alpha0, int* n_sub) {
    if (!p) return REXI_EINVAL;
    for (int k = 0; k < p->K; ++k) {
        if (z) { z[2 * k] = p->z[k].real(); z[2 * k + 1] = p->z[k].imag(); }
        if (alpha) { alpha[2 * k] = p->alpha[k].real(); alpha[2 * k + 1] = p->alpha[k].imag(); }
    }
    if (alpha0) { alpha0[0] = p->alpha0.real(); alpha0[1] = p->alpha0.imag(); }
    if (n_sub) *n_sub = p->n_sub;
    return REXI_OK;
}

int rexi_plan_fcf(const rexi_plan* p, double* sigma, double* beta) {
    if (!p) return REXI_EINVAL;
    for (int k = 0; k < p->K; ++k) {
        if (sigma) { sigma[2 * k] = p->fcf.sigma[k].real(); sigma[2 * k + 1] = p->fcf.sigma[k].imag(); }
        if (beta) { beta[2 * k] = p->fcf.beta[k].real(); beta[2 * k + 1] = p->fcf.beta[k].imag(); }
    }
    return REXI_OK;
}

int rexi_plan_set_potential(rexi_plan* p, const double* V, int on_device, void* stream) {
    if (!p || !V) return REXI_EINVAL;
    DeviceGuard guard(p->device);
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<double> v(p->n);
    if (on_device) {
        if (cudaMemcpyAsync(v.data(), V, sizeof(double) * p->n, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return REXI_ECUDA;
    } else {
        std::memcpy(v.data(), V, sizeof(double) * p->n);
    }
    if (!finite_all(v.data(), v.size())) return REXI_EINVAL;
    p->V.swap(v);
    double vmin = p->V[0], vmax = p->V[0];
    for (double x : p->V) { vmin = std::min(vmin, x); vmax = std::max(vmax, x); }
    int st = upload_diag(p, s, true);
    if (st) return st;
    double lap = 0.0;
    for (int d = 0; d < p->grid.ndim; ++d) lap += 4.0 / (p->h[d] * p->h[d]);
    lap *= p->grid.hbar * p->grid.hbar / (2.0 * p->grid.mass);
    const bool inside = vmin >= p->E_min - 1e-12 * std::fabs(p->E_min) && vmax + lap <= p->E_max + 1e-12 * std::fabs(p->E_max);
    return inside ? REXI_OK : REXI_WACCURACY;
}

int rexi_step(rexi_plan* p, const void* psi_in, void* psi_out, void* stream, rexi_stats* st) {
    if (!p || !psi_in || !psi_out) return REXI_EINVAL;
    DeviceGuard guard(p->device);
    cudaStream_t s = (cudaStream_t)stream;
    if (p->lanczos) {
        int r = lz_launch(p, rexi::LZ_STEP, psi_in, psi_out, s);
        if (r) return p->last_status = r;
        if (!st) return p->last_status = REXI_OK;
        return p->last_status = collect(p, s, p->K, 0, p->K, st, p->n_sub);
    }
    IOArgs io{};
    io.in[0] = (const double2*)psi_in;
    io.out[0] = (double2*)psi_out;
    EngineArgs A = base_args(p, rexi::MODE_STEP, p->fwd, 1, p->n_sub);
    int r = launch(p, A, io, p->fwd.ntiles_items, s);
    if (r) return p->last_status = r;
    if (!st) return p->last_status = REXI_OK;
    return p->last_status = collect(p, s, p->K, 0, p->K, st, p->n_sub);
}

int rexi_cheb_step(rexi_plan* p, const void* psi_in, void* psi_out, double tol, void* stream, int* degree) {
    if (!p || !psi_in || !psi_out) return REXI_EINVAL;
    if (!(tol >= 0.0) || !std::isfinite(tol)) return REXI_EINVAL;
    if (tol == 0.0) tol = 1e-10;
    const double hbar = p->grid.hbar;
    const double R = p->dt * p->W / hbar;
    if (!(p->W > 0.0) || !(p->tau > 0.0) || !std::isfinite(R) || R > 1e6) return REXI_EINVAL;
    // degree: smallest N >= ceil(R) with sum_{k > N} |a_k| <= tol, |a_k| = 2 |J_k(R)|
    const int Lmax = (int)std::ceil(R) + 400;
    const std::vector<double> J = rexi::bessel_j(Lmax, R);
    std::vector<double> tail(Lmax + 2, 0.0);
    for (int k = Lmax; k >= 0; --k) tail[k] = tail[k + 1] + 2.0 * std::fabs(J[k]);
    int N = -1;
    for (int k = (int)std::ceil(R); k < Lmax; ++k)
        if (tail[k + 1] <= tol) { N = k; break; }
    if (N < 0) return REXI_EINVAL;
    // a_k = (2 - delta_k0) (-i)^k J_k(R), times exp(-i dt c / hbar) (centring)
    const std::complex<double> ph = std::exp(std::complex<double>(0.0, -p->dt * p->c / hbar));
    std::vector<double2> coef(N + 1);
    const std::complex<double> mi(0.0, -1.0);
    std::complex<double> ik(1.0, 0.0);
    for (int k = 0; k <= N; ++k) {
        const std::complex<double> a = (k == 0 ? 1.0 : 2.0) * ik * J[k] * ph;
        coef[k] = make_double2(a.real(), a.imag());
        ik *= mi;
    }
    DeviceGuard guard(p->device);
    cudaStream_t s = (cudaStream_t)stream;
    if (N + 1 > p->cheb_cap) {
        if (cudaStreamSynchronize(s) != cudaSuccess) return REXI_ECUDA;
        int r = dalloc(p, &p->d_cheb, (size_t)N + 1);
        if (r) return r;
        p->cheb_cap = N + 1;
    }
    cudaError_t e = cudaMemcpyAsync(p->d_cheb, coef.data(), sizeof(double2) * (N + 1), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->d_bar, 0, 2 * sizeof(unsigned), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->d_err, 0, sizeof(int), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->d_bytes, 0, 3 * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return p->last_status = cuda_fail(e);
    rexi::ChebArgs a{};
    a.prob = p->fwd.d_prob;
    a.psi = (const double2*)psi_in;
    a.out = (double2*)psi_out;
    a.b1 = p->d_tmp0;
    a.b2 = p->d_tmp1;
    a.coef = p->d_cheb;
    a.N = N;
    a.n = p->n;
    a.scale = 1.0 / (p->tau * p->W);
    a.bar = p->d_bar;
    a.err = p->d_err;
    a.timeout_ns = p->timeout_ns;
    a.counters = p->d_bytes;
    const int maxg = rexi::cheb_max_grid(p->device);
    if (maxg <= 0) return p->last_status = REXI_ECUDA;
    const int grid = std::max(1, std::min(maxg, (p->n + rexi::kBlock - 1) / rexi::kBlock));
    e = rexi::launch_cheb(a, grid, s);
    p->last_stream = s;
    p->last_launches = 1;
    p->last_grid = grid;
    if (e != cudaSuccess) return p->last_status = cuda_fail(e);
    if (degree) *degree = N;
    return p->last_status = REXI_OK;
}

int rexi_plan_last_work(rexi_plan* p, double* bytes, double* flops64) {
    if (!p) return REXI_EINVAL;
    DeviceGuard guard(p->device);
    unsigned long long c[2] = {0, 0};
    if (cudaMemcpyAsync(c, p->d_bytes, sizeof(c), cudaMemcpyDeviceToHost, p->last_stream) != cudaSuccess ||
        cudaStreamSynchronize(p->last_stream) != cudaSuccess)
        return REXI_ECUDA;
    if (bytes) *bytes = (double)c[0];
    if (flops64) *flops64 = (double)c[1];
    return REXI_OK;
}

int rexi_step_host(rexi_plan* p, const double* psi_in, double* psi_out, void* stream, rexi_stats* st) {
    if (!p || !psi_in || !psi_out) return REXI_EINVAL;
    DeviceGuard guard(p->device);
    cudaStream_t s = (cudaStream_t)stream;
    const size_t bytes = sizeof(double2) * p->n;
    if (cudaMemcpyAsync(p->d_hin, psi_in, bytes, cudaMemcpyHostToDevice, s) != cudaSuccess) return REXI_ECUDA;
    int r = rexi_step(p, p->d_hin, p->d_hout, stream, st);
    if (r < 0) return r;
    if (cudaMemcpyAsync(psi_out, p->d_hout, bytes, cudaMemcpyDeviceToHost, s) != cudaSuccess) return REXI_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return REXI_ECUDA;
    if (!st) return rexi_plan_last_status(p);
    return r;
}

int rexi_solve_poles(rexi_plan* p, const void* b, void* x, void* stream, rexi_stats* st) {
    if (!p || !b || !x) return REXI_EINVAL;
    DeviceGuard guard(p->device);
    cudaStream_t s = (cudaStream_t)stream;
    if (p->lanczos) {
        int r = lz_launch(p, rexi::LZ_SOLVE, b, x, s);
        if (r) return p->last_status = r;
        if (!st) return p->last_status = REXI_OK;
        return p->last_status = collect(p, s, p->K, 0, p->K, st, 1);
    }
    IOArgs io{};
    io.in[0] = (const double2*)b;
    EngineArgs A = base_args(p, rexi::MODE_SOLVE, p->one, 1, 1);
    int r = launch(p, A, io, p->one.ntiles_items, s);
    if (r) return p->last_status = r;
    cudaError_t e = cudaMemcpyAsync(x, p->d_x, sizeof(double2) * (size_t)p->K * p->n, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return p->last_status = REXI_ECUDA;
    p->last_launches = 1;
    if (!st) return p->last_status = REXI_OK;
    return p->last_status = collect(p, s, p->K, 0, p->K, st, 1);
}

int rexi_apply_poles(rexi_plan* p, const void* v, void* w, void* stream) {
    if (!p || !v || !w) return REXI_EINVAL;
    DeviceGuard guard(p->device);
    cudaError_t e = rexi::launch_apply(p->one.d_prob, p->one.d_items, p->K, (const double2*)v, (double2*)w, p->n,
                                       (cudaStream_t)stream);
    p->last_launches = 1;
    p->last_stream = (cudaStream_t)stream;
    return p->last_status = (e == cudaSuccess ? REXI_OK : REXI_ECUDA);
}

int rexi_pole_sum(rexi_plan* p, const void* psi, const void* x, void* out, void* stream) {
    if (!p || !psi || !x || !out) return REXI_EINVAL;
    DeviceGuard guard(p->device);
    cudaError_t e = rexi::launch_pole_sum(p->one.d_prob, (const double2*)psi, (const double2*)x, (double2*)out,
                                          p->n, p->K, (cudaStream_t)stream);
    p->last_launches = 1;
    p->last_stream = (cudaStream_t)stream;
    return p->last_status = (e == cudaSuccess ? REXI_OK : REXI_ECUDA);
}

int rexi_step_backward(rexi_plan* p, const void* psi_n, const void* grad_out, void* grad_in, double* dLdV,
                       void* stream, rexi_stats* st) {
    if (!p || !psi_n || !grad_out || !grad_in || !dLdV) return REXI_EINVAL;
    DeviceGuard guard(p->device);
    cudaStream_t s = (cudaStream_t)stream;
    int r = ensure_backward(p);
    if (r) return p->last_status = r;
    int launches = 0;
    // forward substeps 0..n_sub-2 from psi_n, saving their outputs as checkpoints
    for (int sub = 0; sub + 1 < p->n_sub; ++sub) {
        IOArgs io{};
        io.in[0] = sub == 0 ? (const double2*)psi_n : p->d_ckpt + (size_t)sub * p->n;
        io.out[0] = p->d_ckpt + (size_t)(sub + 1) * p->n;
        EngineArgs A = base_args(p, rexi::MODE_STEP, p->one, 1, 1);
        r = launch(p, A, io, p->one.ntiles_items, s);
        if (r) return p->last_status = r;
        ++launches;
    }
    IOArgs io{};
    io.in[0] = (const double2*)psi_n;
    io.out[0] = (double2*)grad_in;
    io.gout[0] = (const double2*)grad_out;
    io.dLdV[0] = dLdV;
    EngineArgs A = base_args(p, rexi::MODE_BACKWARD, p->bwd, 1, p->n_sub);
    r = launch(p, A, io, p->bwd.ntiles_items, s);
    if (r) return p->last_status = r;
    p->last_launches = launches + 1;
    if (!st) return p->last_status = REXI_OK;
    return p->last_status = collect(p, s, 2 * p->K, p->K, p->K, st, p->n_sub);
}

int rexi_step_batched(rexi_plan* const* plans, int B, const void* const* psi_in, void* const* psi_out,
                      void* stream, rexi_stats* st) {
    if (!plans || B < 1 || B > rexi::kMaxBatch || !psi_in || !psi_out) return REXI_EINVAL;
    rexi_plan* p0 = plans[0];
    if (!p0) return REXI_EINVAL;
    if (p0->lanczos) {
        // every plan a Lanczos plan on the same device, each plan once
        for (int b = 0; b < B; ++b) {
            rexi_plan* p = plans[b];
            if (!p || !psi_in[b] || !psi_out[b] || !p->lanczos || p->device != p0->device) return REXI_EINVAL;
            for (int c = 0; c < b; ++c)
                if (plans[c] == p) return REXI_EINVAL;
        }
        DeviceGuard guard(p0->device);
        return lz_step_batched(plans, B, psi_in, psi_out, (cudaStream_t)stream, st);
    }
    int total_items = 0, max_sub = 0, total_tiles = 0;
    for (int b = 0; b < B; ++b) {
        rexi_plan* p = plans[b];
        if (!p || !psi_in[b] || !psi_out[b] || p->lanczos) return REXI_EINVAL;
        if (p->device != p0->device || p->fp32 != p0->fp32 || p->m != p0->m ||
            p->opt.ortho != p0->opt.ortho || p->opt.window != p0->opt.window) return REXI_EINVAL;
        const int ng = p->shared ? 1 : 0;
        for (int c = 0; c < b; ++c)
            if (plans[c] == p) return REXI_EINVAL;         // one plan's workspace per problem
        total_items += p->K + ng;
        total_tiles += p->K * ((p->n + p->tile_pole - 1) / p->tile_pole) +
                       ng * ((p->n + p->tile_group - 1) / p->tile_group);
        max_sub = std::max(max_sub, p->n_sub);
    }
    if (total_items > rexi::kMaxItems) return REXI_EINVAL;
    DeviceGuard guard(p0->device);
    cudaStream_t s = (cudaStream_t)stream;

    // Descriptor set of this combination of plans, cached in the first plan and
    // keyed by the plans' process-unique ids and workspace generations (a plan
    // created where a destroyed one lived never matches a stale entry).
    std::vector<unsigned long long> key(B);
    std::vector<int> gens(B);
    for (int b = 0; b < B; ++b) {
        key[b] = plans[b]->uid;
        gens[b] = plans[b]->generation;
    }
    if (p0->batch_key != key || p0->batch_gens != gens || !p0->d_batch_items) {
        std::vector<ProblemDesc> probs;
        std::vector<ItemDesc> items;
        for (int b = 0; b < B; ++b) {
            rexi_plan* p = plans[b];
            const int base = (int)items.size();
            append_items(p, false, b, base, &items);
            probs.push_back(make_problem(p, p->n_sub, base, (int)items.size() - base));
        }
        if (cudaStreamSynchronize(s) != cudaSuccess) return REXI_ECUDA;   // old descriptors may be in use
        int r;
        if (probs.size() > p0->batch_cap_prob) {
            if ((r = dalloc(p0, &p0->d_batch_prob, probs.size()))) return r;
            p0->batch_cap_prob = probs.size();
        }
        if (items.size() > p0->batch_cap_items) {
            if ((r = dalloc(p0, &p0->d_batch_items, items.size()))) return r;
            p0->batch_cap_items = items.size();
        }
        p0->batch_key.clear();                     // invalid until the copies succeed
        if (cudaMemcpy(p0->d_batch_prob, probs.data(), sizeof(ProblemDesc) * probs.size(),
                       cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(p0->d_batch_items, items.data(), sizeof(ItemDesc) * items.size(),
                       cudaMemcpyHostToDevice) != cudaSuccess)
            return REXI_ECUDA;
        p0->batch_key = key;
        p0->batch_gens = gens;
        p0->batch_nitems = (int)items.size();
    }
    IOArgs io{};
    for (int b = 0; b < B; ++b) {
        io.in[b] = (const double2*)psi_in[b];
        io.out[b] = (double2*)psi_out[b];
    }
    DescSet set;
    set.d_prob = p0->d_batch_prob;
    set.d_items = p0->d_batch_items;
    set.nitems = p0->batch_nitems;
    EngineArgs A = base_args(p0, rexi::MODE_STEP, set, B, max_sub);
    // statistics of every plan are zeroed, the barrier/error words are p0's
    for (int b = 1; b < B; ++b)
        if (cudaMemsetAsync(plans[b]->d_stats, 0, sizeof(ItemStats) * (plans[b]->K + plans[b]->ngroups), s) !=
            cudaSuccess)
            return REXI_ECUDA;
    cudaError_t e = cudaMemsetAsync(p0->d_bar, 0, 3 * sizeof(unsigned), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(p0->d_err, 0, sizeof(int), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(p0->d_bytes, 0, 3 * sizeof(unsigned long long), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(p0->d_stats, 0, sizeof(ItemStats) * (p0->K + p0->ngroups), s);
    if (e != cudaSuccess) return REXI_ECUDA;
    const size_t smem = rexi::engine_smem_bytes(A.nitems, p0->fp32, A.ortho);
    const bool wide = !p0->fp32 && p0->ctas_per_sm == 1;
    int maxg = max_grid_cached(p0->fp32, smem, p0->device, wide);
    if (maxg <= 0) return REXI_ECUDA;
    if (p0->ctas_per_sm > 0) maxg = std::min(maxg, p0->ctas_per_sm * sm_count(p0->device));
    const int grid = std::max(1, std::min(maxg, total_tiles));
    e = rexi::launch_engine(p0->fp32, A, io, grid, smem, s, wide);
    for (int b = 0; b < B; ++b) {
        plans[b]->last_stream = s;
        plans[b]->last_launches = 1;
        plans[b]->last_grid = grid;
    }
    if (e != cudaSuccess) return cuda_fail(e);
    if (!st) return REXI_OK;
    int status = REXI_OK;
    unsigned long long nbytes[3] = {0, 0, 0};
    if (cudaMemcpyAsync(nbytes, p0->d_bytes, sizeof(nbytes), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return REXI_ECUDA;
    for (int b = 0; b < B; ++b) {
        rexi_plan* p = plans[b];
        int err = 0;
        std::vector<ItemStats> sv(p->K);
        if (cudaMemcpyAsync(&err, p0->d_err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaMemcpyAsync(sv.data(), p->d_stats, sizeof(ItemStats) * p->K, cudaMemcpyDeviceToHost, s) !=
                cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return REXI_ECUDA;
        rexi_stats& o = st[b];
        std::memset(&o, 0, sizeof(o));
        o.n_sub = p->n_sub;
        bool failed = false;
        for (int k = 0; k < p->K; ++k) {
            if (k < REXI_MAX_POLES) {
                o.iters[k] = sv[k].iters;
                o.cycles[k] = sv[k].cycles;
                o.iters_sq[k] = sv[k].iters_sq;
                o.resid[k] = sv[k].resid;
            }
            o.total_iters += sv[k].iters;
            o.total_cycles += sv[k].cycles;
            o.max_iters_seen = std::max(o.max_iters_seen, sv[k].max_sub_iters);
            failed = failed || sv[k].failed;
        }
        o.status = err ? err : (failed ? REXI_ENOCONV : REXI_OK);
        o.bytes = (double)nbytes[0];
        o.flops64 = (double)nbytes[1];
        o.ops32 = (double)nbytes[2];
        if (o.status != REXI_OK && status == REXI_OK) status = o.status;
        p->last_status = o.status;
    }
    return status;
}

int rexi_plan_last_status(rexi_plan* p) {
    if (!p) return REXI_EINVAL;
    DeviceGuard guard(p->device);
    int err = 0;
    if (cudaMemcpyAsync(&err, p->d_err, sizeof(int), cudaMemcpyDeviceToHost, p->last_stream) != cudaSuccess ||
        cudaStreamSynchronize(p->last_stream) != cudaSuccess)
        return REXI_ECUDA;
    if (err) return err;
    return p->last_status;
}

int rexi_plan_last_launches(const rexi_plan* p) { return p ? p->last_launches : 0; }

int rexi_debug_checks(void) {
#ifdef REXI_DEBUG
    return 1;
#else
    return 0;
#endif
}

int rexi_plan_debug_record(rexi_plan* p, long long rec[4]) {
    if (!p || !rec || !p->d_dbg) return REXI_EINVAL;
    DeviceGuard guard(p->device);
    if (cudaMemcpyAsync(rec, p->d_dbg, 4 * sizeof(long long), cudaMemcpyDeviceToHost, p->last_stream) != cudaSuccess ||
        cudaStreamSynchronize(p->last_stream) != cudaSuccess)
        return REXI_ECUDA;
    return REXI_OK;
}

int rexi_plan_debug_trip(rexi_plan* p, int site) {
    if (!p || !p->d_dbg || site < 0 || site >= rexi::LZ_SITE_COUNT) return REXI_EINVAL;
    p->dbg_trip = site;
    return REXI_OK;
}

int rexi_plan_set_timeout(rexi_plan* p, double seconds) {
    if (!p || !(seconds == seconds) || seconds > 3600.0) return REXI_EINVAL;
    if (seconds <= 0.0) p->timeout_ns = kTimeoutNs;
    else p->timeout_ns = std::max(1ull, (unsigned long long)(seconds * 1e9));
    return REXI_OK;
}

int rexi_plan_set_tiles(rexi_plan* p, int pole_tile, int group_tile, int ctas_per_sm) {
    if (!p) return REXI_EINVAL;
    auto ok = [](int t) { return t >= rexi::kBlock && t <= rexi::kTile && t % rexi::kBlock == 0; };
    if (!ok(pole_tile) || !ok(group_tile) || ctas_per_sm < 0 || ctas_per_sm > 32) return REXI_EINVAL;
    DeviceGuard guard(p->device);
    if (cudaDeviceSynchronize() != cudaSuccess) return REXI_ECUDA;
    if (p->lanczos) {
        // Lanczos plans: group_tile bounds the interior points of a tile,
        // ctas_per_sm the resident CTAs per SM (0: two)
        if (ctas_per_sm > 8) return REXI_EINVAL;
        const int old_target = p->lz_target, old_cps = p->lz_cps;
        p->lz_target = group_tile;
        p->lz_cps = ctas_per_sm > 0 ? ctas_per_sm : 2;
        const int r = lz_configure(p);
        if (r) {
            p->lz_target = old_target;
            p->lz_cps = old_cps;
            lz_configure(p);
            return r;
        }
    }
    p->tile_pole = pole_tile;
    p->tile_group = group_tile;
    p->ctas_per_sm = ctas_per_sm;
    p->generation++;                              // batched descriptor caches rebuild
    return build_sets(p);
}

int rexi_plan_set_trace(rexi_plan* p, int capacity) {
    if (!p || capacity < 0) return REXI_EINVAL;
    DeviceGuard guard(p->device);
    if (capacity > p->trace_cap) {
        int st = dalloc(p, &p->d_trace, (size_t)1 + 2 * (size_t)capacity);
        if (st) return st;
        if (cudaMemset(p->d_trace, 0, sizeof(unsigned long long)) != cudaSuccess) return REXI_ECUDA;
    }
    p->trace_cap = capacity;
    return REXI_OK;
}

int rexi_plan_set_cta_trace(rexi_plan* p, int phases) {
    if (!p || phases < 0) return REXI_EINVAL;
    DeviceGuard guard(p->device);
    const int stride = 8 * sm_count(p->device);          // no more than 8 CTAs of 256 threads per SM
    if (phases > 0 && (phases > p->cta_trace_phases || stride != p->cta_trace_stride)) {
        int st = dalloc(p, &p->d_cta_trace, (size_t)1 + (size_t)phases * (size_t)stride);
        if (st) return st;
        if (cudaMemset(p->d_cta_trace, 0, sizeof(unsigned long long)) != cudaSuccess) return REXI_ECUDA;
        p->cta_trace_stride = stride;
    }
    p->cta_trace_phases = phases;
    return REXI_OK;
}

int rexi_plan_read_cta_trace(rexi_plan* p, long long* out, int cap, int* grid) {
    if (!p || (cap > 0 && !out)) return REXI_EINVAL;
    if (grid) *grid = p->last_grid;
    if (p->cta_trace_phases <= 0 || !p->d_cta_trace || p->last_grid <= 0) return 0;
    DeviceGuard guard(p->device);
    unsigned long long count = 0;
    if (cudaStreamSynchronize(p->last_stream) != cudaSuccess ||
        cudaMemcpy(&count, p->d_cta_trace, sizeof(count), cudaMemcpyDeviceToHost) != cudaSuccess)
        return REXI_ECUDA;
    const int g = std::min(p->last_grid, p->cta_trace_stride);
    const long long rows = std::min<long long>((long long)count, std::min<long long>(p->cta_trace_phases, cap / g));
    for (long long r = 0; r < rows; ++r)
        if (cudaMemcpy(out + r * g, p->d_cta_trace + 1 + r * p->cta_trace_stride, sizeof(long long) * g,
                       cudaMemcpyDeviceToHost) != cudaSuccess)
            return REXI_ECUDA;
    return (int)count;
}

int rexi_plan_read_trace(rexi_plan* p, long long* out, int cap) {
    if (!p || (cap > 0 && !out)) return REXI_EINVAL;
    if (p->trace_cap <= 0 || !p->d_trace) return 0;
    DeviceGuard guard(p->device);
    unsigned long long count = 0;
    if (cudaStreamSynchronize(p->last_stream) != cudaSuccess ||
        cudaMemcpy(&count, p->d_trace, sizeof(count), cudaMemcpyDeviceToHost) != cudaSuccess)
        return REXI_ECUDA;
    const int n = (int)std::min<unsigned long long>(count, (unsigned long long)std::min(cap, p->trace_cap));
    if (n > 0 && cudaMemcpy(out, p->d_trace + 1, sizeof(long long) * 2 * n, cudaMemcpyDeviceToHost) != cudaSuccess)
        return REXI_ECUDA;
    return (int)count;
}

}  // extern "C"
