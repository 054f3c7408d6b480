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
// bar[1] = generation.  partials: [kSlots][kMaxTeam][kVals] doubles.
constexpr int kMaxTeam = 1024;
constexpr int kSlots = 4;
constexpr int kVals = 4;

struct Team {
    int rank;          // CTA rank within the team
    int size;          // number of CTAs in the team
    unsigned* bar;     // 2 words, zero-initialised
    int* status;       // shared device status word (hmc_status, 0 = ok)
    double* partials;  // kSlots * kMaxTeam * kVals
    int slot;          // rotating partials slot (identical on all CTAs)
};

__device__ __forceinline__ bool team_failed(const Team& tm) {
    return *((volatile int*)tm.status) != 0;
}

__device__ __forceinline__ void set_status(int* status, int code) {
    atomicCAS(status, 0, code);
}

// Bounded generation barrier over the team.  Returns false (on every
// thread of the CTA) if the team's status is set or the wait timed out.
__device__ inline bool team_barrier(Team& tm) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        if (tm.size > 1) {
            cuda::atomic_ref<unsigned, cuda::thread_scope_device> cnt(tm.bar[0]);
            cuda::atomic_ref<unsigned, cuda::thread_scope_device> gen(tm.bar[1]);
            __threadfence();
            const unsigned g = gen.load(cuda::memory_order_acquire);
            if (cnt.fetch_add(1u, cuda::memory_order_acq_rel) == (unsigned)(tm.size - 1)) {
                cnt.store(0u, cuda::memory_order_relaxed);
                gen.store(g + 1u, cuda::memory_order_release);
            } else {
                const uint64_t t0 = global_ns();
                unsigned ns = 32;
                while (gen.load(cuda::memory_order_acquire) == g) {
                    __nanosleep(ns);
                    if (ns < 256) ns <<= 1;
                    if (team_failed(tm)) { ok = 0; break; }
                    if (global_ns() - t0 > kWaitLimitNs) {
                        set_status(tm.status, HMC_ERR_TIMEOUT);
                        ok = 0;
                        break;
                    }
                }
            }
            __threadfence();
        }
        if (team_failed(tm)) ok = 0;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
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

// Deterministic team-wide sum of NV values: every CTA of the team gets the
// same bits (each sums the per-CTA partials in the same fixed order).
// Contains a team barrier; returns false if the team failed.
template <int NV>
__device__ inline bool team_sum(Team& tm, double (&v)[NV]) {
    static_assert(NV <= kVals, "too many values");
    __shared__ double s_out[NV];
    block_reduce<NV>(v);
    double* part = tm.partials + (size_t)tm.slot * kMaxTeam * kVals;
    if (threadIdx.x == 0)
#pragma unroll
        for (int j = 0; j < NV; ++j) part[tm.rank * kVals + j] = v[j];
    tm.slot = (tm.slot + 1) % kSlots;
    if (!team_barrier(tm)) return false;
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
#pragma unroll
        for (int j = 0; j < NV; ++j) {
            double a = 0.0;
            for (int r = lane; r < tm.size; r += 32) a += ((volatile double*)part)[r * kVals + j];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
            if (lane == 0) s_out[j] = a;
        }
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < NV; ++j) v[j] = s_out[j];
    __syncthreads();
    return true;
}

__device__ __forceinline__ bool finite_d(double a) { return isfinite(a); }

}  // namespace hmc
