// Device primitives shared by the persistent kernels: a bounded grid barrier
// for co-resident (cooperative) grids, acquire/release accesses, the global
// timer, and an integer-only FP64 -> FP32 conversion for inner products.
#pragma once

#include <cuda_runtime.h>

namespace rexi {
namespace dev {

constexpr int kErrTimeout = -5;   // REXI_ETIMEOUT

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int ld_relaxed_s32(const int* p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

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

// ---- bulk copies global -> shared with completion on an mbarrier -----------

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned long long* b, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
// Makes the initialised mbarrier visible to the asynchronous proxy.
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
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
// Global to shared copy of `bytes` (a multiple of 16, both addresses 16-byte
// aligned) whose completion is counted on mbarrier b.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* b) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(b))
                 : "memory");
}
// Orders this thread's earlier generic-proxy accesses (and those it has
// acquired) before its later bulk copies.
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async;" ::: "memory"); }

// Bounded wait for phase `parity` of mbarrier b.  On expiry the sticky error
// word is set and a second wait (at least 10 ms) lets copies still in flight
// land before the buffer is reused or the CTA leaves; the launch then ends at
// its next grid barrier.
__device__ __forceinline__ bool mbar_wait(unsigned long long* b, unsigned parity, int* err,
                                          unsigned long long timeout_ns) {
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

// All `count` CTAs that share `bar` (a co-resident grid, or one problem's range
// of CTAs in a batched launch) meet here.  bar[0] counts arrivals and is zeroed
// before every launch; `gen` is the calling CTA's count of barriers passed
// (thread 0's copy is the one used).  Every CTA adds one to bar[0] with a
// release reduction -- after the CTA barrier, it orders all of the CTA's
// earlier writes before the arrival -- and then waits with acquire loads until
// the count reaches gen x count: every arrival is a release heading a release
// sequence that contains the later arrivals, so reading the final count
// synchronises with all of them, and no CTA has to publish for the others.
// Every wait is bounded by timeout_ns: on expiry the sticky error word is set.
// A wait also ends when another CTA has set the error word (it may have left
// the kernel and never arrive).  The function returns false whenever the error
// word is set, so every CTA leaves the kernel at its next barrier.
// Bounded wait (thread 0 of a CTA) until the arrival count *bar reaches
// target.  Each poll reads the sticky error word (relaxed) and then the count
// (acquire): the acquire orders only later accesses, so both loads are in
// flight together (one L2 round trip per poll), and the acquire load that
// observes the final count synchronises with the release arrivals.  The wait
// also ends when the error word is set; on expiry it sets it.  Returns whether
// the error word was clear at the last poll.
__device__ __forceinline__ bool wait_count(const unsigned* bar, unsigned target, int* err,
                                           unsigned long long timeout_ns) {
    const unsigned long long t0 = global_ns();
    for (;;) {
        const int e = ld_relaxed_s32(err);
        const unsigned v = ld_acquire_u32(bar);
        if (e != 0) return false;
        if ((int)(v - target) >= 0) return true;
        if (global_ns() - t0 > timeout_ns) {
            atomicExch(err, kErrTimeout);
            return false;
        }
    }
}

// Grid barrier of `count` co-resident CTAs: thread 0 arrives with a release
// reduction on the arrival count (gen: barriers this CTA has passed) and
// polls it; the CTA learns the outcome through shared memory, so no other
// thread reads global memory for it.  Returns false when the launch must end
// (an error or a timeout anywhere: a CTA that passed the barrier before the
// error word was set stops at its next barrier).
__device__ __forceinline__ bool grid_sync(unsigned* bar, unsigned count, unsigned& gen, int* err,
                                          unsigned long long timeout_ns) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        gen += 1u;
        const unsigned target = gen * count;
        asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(bar) : "memory");
        ok = wait_count(bar, target, err, timeout_ns) ? 1 : 0;
    }
    __syncthreads();
    return ok != 0;
}

}  // namespace dev
}  // namespace rexi
