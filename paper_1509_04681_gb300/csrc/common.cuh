// Shared device/host helpers of the CGGM CUDA library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <cstdio>

#include "../../include/cggm.h"

namespace cggm {

// Device status word codes (written by kernels, read by the host after a launch).
enum DevErr : int {
    DEV_OK = 0,
    DEV_NOTPD = 1,       // Cholesky pivot <= 0 or not finite
    DEV_TIMEOUT = 2,     // a grid barrier exceeded its deadline
    DEV_NONFINITE = 3,   // NaN/Inf met in a coordinate step
    DEV_BADINDEX = 4,    // an index outside its matrix
};

struct Status {
    cggm_status code = CGGM_OK;
    explicit operator bool() const { return code == CGGM_OK; }
};

#define CGGM_CUDA_TRY(expr)                                                              \
    do {                                                                                 \
        cudaError_t _e = (expr);                                                         \
        if (_e != cudaSuccess) {                                                         \
            if (getenv("CGGM_DEBUG"))                                                    \
                fprintf(stderr, "cggm: %s failed at %s:%d: %s\n", #expr, __FILE__,       \
                        __LINE__, cudaGetErrorString(_e));                               \
            return _e == cudaErrorMemoryAllocation ? CGGM_ENOMEM : CGGM_ECUDA;           \
        }                                                                                \
    } while (0)

#define CGGM_TRY(expr)                                                                   \
    do {                                                                                 \
        cggm_status _s = (expr);                                                         \
        if (_s != CGGM_OK) return _s;                                                    \
    } while (0)

inline unsigned ceil_div(int64_t a, int64_t b) { return (unsigned)((a + b - 1) / b); }

// Number of SMs of the current device (looked up once per device).
int sm_count();

// Host-side count of kernel launches issued by this library (all contexts, process-wide);
// reported per call in cggm_info.launches.
int64_t &launch_counter();
inline void note_launch() { __atomic_add_fetch(&launch_counter(), 1, __ATOMIC_RELAXED); }

// ---------------------------------------------------------------------------------
// Grid-wide barrier for persistent kernels launched cooperatively (all CTAs resident).
// Sense/generation based, acquire/release ordered, with a wall-clock deadline: a CTA
// that waits longer than `deadline_ns` sets the error word to DEV_TIMEOUT; every
// waiter also leaves as soon as the error word is nonzero.  Returns false on error.
// ---------------------------------------------------------------------------------
struct GridBarrier {
    unsigned long long arrived;  // arrivals since the launch (zeroed before it); monotonic
    // pipelined coordinate passes (sweeps.cu), all monotonic from zero: batches whose steps
    // CTA 0 has published, and the phase-A and phase-C completions of the other CTAs (one
    // per CTA and batch)
    unsigned long long mu_ready, a_done, c_done;
};

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ int ld_acquire_int(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// Grid-wide barrier of a cooperative launch, in two halves so that a CTA can issue loads
// between its arrival and its wait.  Every CTA passes the barriers of a launch in the same
// order and counts them itself (`round`, from 0): its arrival adds one to a counter that
// only grows, as a release reduction that returns nothing (so the arrival costs no round
// trip), and its wait lasts until the counter reaches (round + 1) nblocks.  A wait that
// exceeds deadline_ns, or sees another CTA's error, returns false (and records DEV_TIMEOUT
// in the first case).
struct GridTicket {
    unsigned long long target;  // thread 0: the count that ends this round
};

__device__ __forceinline__ void red_release_add(unsigned long long *p, unsigned long long v) {
    asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ GridTicket grid_arrive(GridBarrier *bar, unsigned nblocks,
                                                  unsigned &round) {
    __syncthreads();  // the CTA's work of this round is done (and ordered before the release)
    GridTicket t{0};
    if (threadIdx.x == 0) {
        red_release_add(&bar->arrived, 1ull);
        t.target = (unsigned long long)(round + 1) * nblocks;
    }
    round++;
    return t;
}

__device__ __forceinline__ bool grid_wait(GridBarrier *bar, int *err, GridTicket t,
                                          uint64_t deadline_ns = 2000000000ull) {
    __shared__ int s_ok;
    if (threadIdx.x == 0) {
        int ok = 1;
        const uint64_t t0 = global_ns();
        unsigned spins = 0;
        while (ld_acquire_u64(&bar->arrived) < t.target) {
            if ((++spins & 63u) == 0) {
                if (ld_acquire_int(err) != 0) { ok = 0; break; }
                if (global_ns() - t0 > deadline_ns) {
                    atomicCAS(err, 0, (int)DEV_TIMEOUT);
                    ok = 0;
                    break;
                }
            }
        }
        if (ok && ld_acquire_int(err) != 0) ok = 0;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Every thread of the CTA: waits (thread 0 polls, acquire) until *c1 >= t1 and, when c2 is
// given, *c2 >= t2; bounded by deadline_ns, and left early when the error word is nonzero.
// Returns false on failure (DEV_TIMEOUT recorded when the deadline passed).
__device__ __forceinline__ bool cta_wait_counts(const unsigned long long *c1,
                                                unsigned long long t1,
                                                const unsigned long long *c2,
                                                unsigned long long t2, int *err,
                                                uint64_t deadline_ns = 2000000000ull) {
    __shared__ int s_ok;
    if (threadIdx.x == 0) {
        int ok = 1;
        const uint64_t t0 = global_ns();
        unsigned spins = 0;
        while (ld_acquire_u64(c1) < t1 || (c2 && ld_acquire_u64(c2) < t2)) {
            if ((++spins & 63u) == 0) {
                if (ld_acquire_int(err) != 0) { ok = 0; break; }
                if (global_ns() - t0 > deadline_ns) {
                    atomicCAS(err, 0, (int)DEV_TIMEOUT);
                    ok = 0;
                    break;
                }
            }
        }
        if (ok && ld_acquire_int(err) != 0) ok = 0;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Thread 0, after a __syncthreads that ends the CTA's part of a step: counts it (release).
__device__ __forceinline__ void cta_count(unsigned long long *c) {
    if (threadIdx.x == 0) red_release_add(c, 1ull);
}

__device__ __forceinline__ bool grid_sync(GridBarrier *bar, int *err, unsigned nblocks,
                                          unsigned &round, uint64_t deadline_ns = 2000000000ull) {
    return grid_wait(bar, err, grid_arrive(bar, nblocks, round), deadline_ns);
}

// Warp reductions
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block reduction of a double (blockDim multiple of 32, <= 1024); result valid in all
// threads.
__device__ __forceinline__ double block_sum(double v) {
    __shared__ double s_part[32];
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) s_part[w] = v;
    __syncthreads();
    const int nw = (blockDim.x + 31) >> 5;
    double r = (threadIdx.x < nw) ? s_part[threadIdx.x] : 0.0;
    if (w == 0) r = warp_sum(r);
    __shared__ double s_res;
    if (threadIdx.x == 0) s_res = r;
    __syncthreads();
    return s_res;
}

__device__ __forceinline__ double soft_threshold(double w, double r) {
    return w > r ? w - r : (w < -r ? w + r : 0.0);
}

}  // namespace cggm
