// common.cuh -- device utilities shared by the library's kernels:
// complex helpers, the Philox4x32-10 generator, a bounded team barrier and
// deterministic team reductions.
#pragma once

#include <cuda_runtime.h>
#include <cuda/atomic>
#include <stdint.h>

#include "../../include/hmc.h"

namespace hmc {

// ---------------------------------------------------------------- complex
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cmulc(double2 a, double2 b) {  // conj(a) * b
    return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cmulcf(float2 a, float2 b) {
    return make_float2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}

// ---------------------------------------------------------------- Philox
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of the
// 4x32 bijection, key bumped by the Weyl constants between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k.x += 0x9E3779B9u;
            k.y += 0xBB67AE85u;
        }
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

enum : uint32_t { kStreamMomentum = 0, kStreamNoise = 1, kStreamMetropolis = 2 };

// Counter (element, stream, trajectory mod 2^32, chain), key = seed halves.
__device__ __forceinline__ uint4 philox_draw(uint64_t seed, uint32_t stream, uint64_t traj,
                                             uint32_t chain, uint32_t e) {
    return philox4x32_10(make_uint4(e, stream, (uint32_t)traj, chain),
                         make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
}

// Two uniforms in (0,1) from 53-bit integers: ((hi<<32|lo) >> 11) + 1/2, * 2^-53.
__device__ __forceinline__ double2 uniform_pair(uint4 r) {
    const uint64_t a = ((((uint64_t)r.x) << 32) | r.y) >> 11;
    const uint64_t b = ((((uint64_t)r.z) << 32) | r.w) >> 11;
    const double s = 1.1102230246251565e-16;  // 2^-53
    return make_double2(((double)a + 0.5) * s, ((double)b + 0.5) * s);
}

// Box-Muller: (sqrt(-2 ln u1) cos(2 pi u2), sqrt(-2 ln u1) sin(2 pi u2)).
__device__ __forceinline__ double2 normal_pair(uint4 r) {
    const double2 u = uniform_pair(r);
    const double rad = sqrt(-2.0 * log(u.x));
    double sn, cs;
    sincospi(2.0 * u.y, &sn, &cs);
    return make_double2(rad * cs, rad * sn);
}

// ---------------------------------------------------------------- timers
__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Every spin in this library gives up after this long and records
// HMC_ERR_TIMEOUT instead of waiting forever.
constexpr uint64_t kWaitLimitNs = 20ull * 1000ull * 1000ull * 1000ull;  // 20 s

// ---------------------------------------------------------------- team
// A team is a set of co-resident CTAs of one persistent (cooperative)
// launch that work on one Markov chain.  bar[0] = arrival count,
// bar[1] = generation.  partials: per-CTA partial sums [kMaxTeam][kVals],
// followed by the published team totals [kVals].
constexpr int kMaxTeam = 1024;
constexpr int kVals = 4;
constexpr int kSlots = 1;          // partial-sum buffers (one suffices, see team_sum)
constexpr size_t kPartialDoubles = (size_t)kMaxTeam * kVals + kVals;

struct Team {
    int rank;          // CTA rank within the team
    int size;          // number of CTAs in the team
    unsigned* bar;     // 2 words, zero-initialised
    int* status;       // shared device status word (hmc_status, 0 = ok)
    double* partials;  // kPartialDoubles
    int slot;          // unused (kept for layout stability)
};

__device__ __forceinline__ bool team_failed(const Team& tm) {
    return *((volatile int*)tm.status) != 0;
}

__device__ __forceinline__ void set_status(int* status, int code) {
    atomicCAS(status, 0, code);
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Fixed-order CTA reduction of NV doubles; result valid on thread 0.
template <int NV>
__device__ __forceinline__ void block_reduce(double (&v)[NV]) {
    __shared__ double s_red[32][NV];
#pragma unroll
    for (int j = 0; j < NV; ++j)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[j] += __shfl_down_sync(0xffffffffu, v[j], o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int j = 0; j < NV; ++j) s_red[warp][j] = v[j];
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int j = 0; j < NV; ++j) {
            double a = lane < nw ? s_red[lane][j] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
            v[j] = a;
        }
    }
}

// Team barrier fused with a deterministic sum of NV values (NV = 0: plain
// barrier).  Every CTA writes its partials, then arrives on the counter; the
// last CTA to arrive sums the partials of all ranks in rank order (a fixed
// order, so every run and every CTA gets the same bits), publishes the
// totals and flips the generation word; the others spin (bounded) on the
// generation and read the totals.  One buffer suffices: a CTA can write its
// next partials only after passing this barrier, and the last arriver has
// read every partial before it releases the barrier.
// Returns false on every thread of the CTA if the team failed or a wait
// timed out.
template <int NV>
__device__ inline bool team_sync(Team& tm, double* v) {
    __shared__ int s_ok;
    __shared__ int s_last;
    __shared__ double s_out[NV > 0 ? NV : 1];
    if constexpr (NV > 0) block_reduce<NV>(*reinterpret_cast<double(*)[NV]>(v));
    if (tm.size == 1) {
        if (threadIdx.x == 0) {
#pragma unroll
            for (int j = 0; j < NV; ++j) s_out[j] = v[j];
            s_ok = !team_failed(tm);
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < NV; ++j) v[j] = s_out[j];
        const int ok = s_ok;
        __syncthreads();
        return ok != 0;
    }
    double* totals = tm.partials + (size_t)kMaxTeam * kVals;
    cuda::atomic_ref<unsigned, cuda::thread_scope_device> cnt(tm.bar[0]);
    cuda::atomic_ref<unsigned, cuda::thread_scope_device> gen(tm.bar[1]);
    unsigned g = 0;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int j = 0; j < NV; ++j) tm.partials[tm.rank * kVals + j] = v[j];
        g = gen.load(cuda::memory_order_relaxed);
        __threadfence();
        s_last = cnt.fetch_add(1u, cuda::memory_order_acq_rel) == (unsigned)(tm.size - 1);
    }
    __syncthreads();
    if (s_last) {
        // last arriver: fixed-order sum of all partials by warp 0, publish
        if (NV > 0 && threadIdx.x < 32) {
            __threadfence();
            const int lane = threadIdx.x;
#pragma unroll
            for (int j = 0; j < NV; ++j) {
                double a = 0.0;
                for (int r = lane; r < tm.size; r += 32)
                    a += ((volatile double*)tm.partials)[r * kVals + j];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
                if (lane == 0) {
                    totals[j] = a;
                    s_out[j] = a;
                }
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            cnt.store(0u, cuda::memory_order_relaxed);
            __threadfence();
            gen.store(g + 1u, cuda::memory_order_release);
            s_ok = !team_failed(tm);
        }
    } else if (threadIdx.x == 0) {
        int ok = 1;
        const uint64_t t0 = global_ns();
        for (unsigned n = 1; ld_acquire_u32(&tm.bar[1]) == g; ++n) {
            if ((n & 1023u) == 0) {
                if (team_failed(tm)) { ok = 0; break; }
                if (global_ns() - t0 > kWaitLimitNs) {
                    set_status(tm.status, HMC_ERR_TIMEOUT);
                    ok = 0;
                    break;
                }
            }
        }
        __threadfence();
#pragma unroll
        for (int j = 0; j < NV; ++j) s_out[j] = ((volatile double*)totals)[j];
        s_ok = ok && !team_failed(tm);
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < NV; ++j) v[j] = s_out[j];
    const int ok = s_ok;
    __syncthreads();
    return ok != 0;
}

__device__ inline bool team_barrier(Team& tm) { return team_sync<0>(tm, nullptr); }

template <int NV>
__device__ inline bool team_sum(Team& tm, double (&v)[NV]) {
    return team_sync<NV>(tm, v);
}

__device__ __forceinline__ bool finite_d(double a) { return isfinite(a); }

}  // namespace hmc
