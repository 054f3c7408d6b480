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

enum : uint32_t { kStreamMomentum = 0, kStreamNoise = 1, kStreamMetropolis = 2,
                  kStreamHeavy = 3,     // the heavy pseudofermion of mass preconditioning
                  kStreamZ2 = 4 };      // Z2 noise of the stochastic trace estimates

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

// Every spin in this library gives up after a time limit and records
// HMC_ERR_TIMEOUT instead of waiting forever.  The limit lives in the
// status block next to the status word: int status, int (unused), uint64
// limit in ns at byte offset 8; zero there selects the default below.
constexpr uint64_t kWaitLimitNs = 20ull * 1000ull * 1000ull * 1000ull;  // 20 s
constexpr size_t kStatusBlockBytes = 16;
__device__ __forceinline__ uint64_t wait_limit_ns(const int* status) {
    const uint64_t v = *reinterpret_cast<const volatile uint64_t*>(status + 2);
    return v ? v : kWaitLimitNs;
}

// ---------------------------------------------------------------- team
// A team is a set of co-resident CTAs of one persistent (cooperative)
// launch that work on one Markov chain.  bar[0] = arrival count,
// bar[1] = generation.  partials: per-CTA partial sums [kMaxTeam][kVals],
// followed by the published team totals [kVals].
constexpr int kMaxTeam = 1024;
constexpr int kVals = 4;
constexpr int kSlots = 1;          // partial-sum buffers (one suffices, see team_sum)
constexpr size_t kPartialDoubles = (size_t)kMaxTeam * kVals + kVals;

// Synchronisation state of a team that is one thread-block cluster: every
// CTA pushes its partial sums into every member's slot (distributed shared
// memory) and arrives on every member's mbarrier; each CTA then waits on its
// own mbarrier only.  Sync k uses barrier and slots k & 1: a member can only
// start sync k+2 after every member has arrived for k+1, which each does
// after finishing its wait (and reads) of sync k, so an early arrival for
// the next sync never lands on the barrier a CTA is still waiting on, and a
// slot is never rewritten while it may still be read.
constexpr int kMaxCluster = 16;
struct ClusterSync {
    uint64_t bar[2];                       // one arrival per member per sync
    unsigned count;                        // syncs this CTA has completed
    double part[2][kMaxCluster][kVals];    // FP64 sums: [k & 1][member][value]
    float part_f[2][kMaxCluster];          // FP32 sums: [k & 1][member]
    // Byte-counted exchanges (st.async / bulk copies with mbarrier
    // complete_tx): phase k uses bar_tx[k & 1], armed by this CTA's own
    // arrive.expect_tx; the data itself completes the phase, so the senders
    // need no release fence.
    uint64_t bar_tx[2];
    unsigned count_tx;
    float part_tx[2][kMaxCluster];
};

struct Team {
    int rank;          // CTA rank within the team
    int size;          // number of CTAs in the team
    unsigned* bar;     // 2 words, zero-initialised
    int* status;       // shared device status word (hmc_status, 0 = ok)
    double* partials;  // kPartialDoubles
    ClusterSync* cs;   // non-null: the team is this CTA's cluster, rank = cluster rank
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

__device__ __forceinline__ uint32_t cta_smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint32_t cluster_ctarank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// Hardware barrier over every thread of the cluster (all threads call it).
__device__ __forceinline__ void cluster_barrier_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\t"
                 "barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Set up the cluster team state; all threads of every member call it before
// the first cluster sync.  Ends with a hardware cluster barrier, so no
// member arrives remotely on a barrier that is not yet initialised.
__device__ inline void cluster_sync_init(ClusterSync* cs, int size) {
    if (threadIdx.x == 0) {
        for (int b = 0; b < 2; ++b) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(cta_smem_u32(&cs->bar[b])),
                         "r"(size)
                         : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(
                             cta_smem_u32(&cs->bar_tx[b]))
                         : "memory");
        }
        cs->count = 0;
        cs->count_tx = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    cluster_barrier_all();
}

// Warp 0 of a cluster team, sync k = cs->count: lane r < size stores this
// CTA's NV values (FP64 in `part`, or one FP32 in `part_f` when F32) into
// member r's slot and arrives on member r's barrier k & 1 (release: orders
// this CTA's earlier writes, shared and global, local and remote, before the
// arrival).
template <int NV, bool F32>
__device__ inline void cluster_push(const Team& tm, const double* v, float vf) {
    ClusterSync* cs = tm.cs;
    const int par = (int)(cs->count & 1u);
    const int lane = threadIdx.x & 31;
    if (lane < tm.size) {
        const uint32_t r = (uint32_t)lane;
        uint32_t rs, rb;
        if constexpr (F32) {
            asm volatile("mapa.shared::cluster.u32 %0, %1, %2;"
                         : "=r"(rs)
                         : "r"(cta_smem_u32(&cs->part_f[par][tm.rank])), "r"(r));
            asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(rs), "f"(vf) : "memory");
        } else {
            asm volatile("mapa.shared::cluster.u32 %0, %1, %2;"
                         : "=r"(rs)
                         : "r"(cta_smem_u32(&cs->part[par][tm.rank][0])), "r"(r));
#pragma unroll
            for (int j = 0; j < NV; ++j)
                asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(rs + 8 * j), "d"(v[j])
                             : "memory");
        }
        asm volatile("mapa.shared::cluster.u32 %0, %1, %2;"
                     : "=r"(rb)
                     : "r"(cta_smem_u32(&cs->bar[par])), "r"(r));
        asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(rb)
                     : "memory");
    }
}

// Lane 0 of a cluster team: wait (bounded, acquire) until every member has
// arrived for sync cs->count.  False on timeout or team failure.  No global
// memory is touched unless the wait runs long.
__device__ inline bool cluster_wait(const Team& tm) {
    ClusterSync* cs = tm.cs;
    const unsigned k = cs->count;
    const uint32_t bar = cta_smem_u32(&cs->bar[k & 1u]);
    const uint32_t phase = (k >> 1) & 1u;
    uint64_t t0 = 0;
    for (unsigned n = 1;; ++n) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.test_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(bar), "r"(phase)
            : "memory");
        if (done) return true;
        if ((n & 1023u) == 0) {
            if (t0 == 0) t0 = global_ns();
            if (team_failed(tm)) return false;
            if (global_ns() - t0 > wait_limit_ns(tm.status)) {
                set_status(tm.status, HMC_ERR_TIMEOUT);
                return false;
            }
        }
    }
}

// Warp 0: push, then lane 0 waits.  Result valid on lane 0.
template <int NV, bool F32>
__device__ inline bool cluster_push_wait(const Team& tm, const double* v, float vf) {
    cluster_push<NV, F32>(tm, v, vf);
    if ((threadIdx.x & 31) != 0) return true;
    return cluster_wait(tm);
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
// kPre: the CTA's values are already summed and valid on thread 0 only.
// kF32: the values are FP32 numbers (held exactly in the doubles) and the
// team sum is formed in FP32, in the order of the cluster path.
template <int NV, bool kPre = false, bool kF32 = false>
__device__ inline bool team_sync(Team& tm, double* v) {
    __shared__ int s_ok;
    __shared__ int s_last;
    __shared__ double s_out[NV > 0 ? NV : 1];
    if constexpr (NV > 0 && !kPre) block_reduce<NV>(*reinterpret_cast<double(*)[NV]>(v));
    if (tm.size == 1) {
        if (threadIdx.x == 0) {
#pragma unroll
            for (int j = 0; j < NV; ++j) s_out[j] = v[j];
            s_ok = 1;
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < NV; ++j) v[j] = s_out[j];
        const int ok = s_ok;
        __syncthreads();
        return ok != 0;
    }
    if (tm.cs) {
        // cluster team: same summation order as the global path below
        // (lane r holds member r's partial, then a fixed shuffle tree)
        if (threadIdx.x < 32) {
            double pv[NV > 0 ? NV : 1];
#pragma unroll
            for (int j = 0; j < NV; ++j) pv[j] = __shfl_sync(0xffffffffu, v[j], 0);
            const bool ok = cluster_push_wait<NV, false>(tm, pv, 0.f);
            if (threadIdx.x == 0) {
                s_last = (int)(tm.cs->count & 1u);
                tm.cs->count += 1u;
                s_ok = ok ? 1 : 0;
            }
        }
        __syncthreads();
        if (NV > 0 && threadIdx.x < 32) {
            const int par = s_last, lane = threadIdx.x;
#pragma unroll
            for (int j = 0; j < NV; ++j) {
                double a = lane < tm.size ? tm.cs->part[par][lane][j] : 0.0;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
                if (lane == 0) s_out[j] = a;
            }
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
                if constexpr (kF32) {
                    float a = 0.f;
                    for (int r = lane; r < tm.size; r += 32)
                        a += (float)((volatile double*)tm.partials)[r * kVals + j];
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
                    if (lane == 0) {
                        totals[j] = (double)a;
                        s_out[j] = (double)a;
                    }
                } else {
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
                if (global_ns() - t0 > wait_limit_ns(tm.status)) {
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

// Team sum of one FP32 value per thread, in FP32 throughout (the inner CG
// loop's norms): warps reduce with a fixed shuffle tree, thread 0 adds the
// warp sums in warp order, members' sums are added in rank order.  No FP64
// arithmetic (slow on this part) and, for a one-CTA or cluster team, no
// global memory.  Result on every thread.
__device__ inline bool team_sum_f(Team& tm, float x, float& out) {
    __shared__ float s_w[32];
    __shared__ float s_tot;
    __shared__ int s_fok;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    if (lane == 0) s_w[warp] = x;
    __syncthreads();
    if (tm.size > 1 && !tm.cs) {
        // global-memory team: the CTAs' FP32 sums, added in FP32 in the
        // order of the cluster path (same bits for the same team)
        double v[1] = {0.0};
        if (threadIdx.x == 0) {
            float a = 0.f;
            for (int w = 0; w < nw; ++w) a += s_w[w];
            v[0] = (double)a;
        }
        const bool ok = team_sync<1, true, true>(tm, v);
        out = (float)v[0];
        return ok;
    }
    if (warp == 0) {
        float a = 0.f;
        if (lane == 0)
            for (int w = 0; w < nw; ++w) a += s_w[w];
        a = __shfl_sync(0xffffffffu, a, 0);
        if (tm.size == 1) {
            if (lane == 0) {
                s_tot = a;
                s_fok = 1;
            }
        } else {
            const bool ok = cluster_push_wait<1, true>(tm, nullptr, a);
            const int par = (int)(tm.cs->count & 1u);
            __syncwarp();
            float b = lane < tm.size ? tm.cs->part_f[par][lane] : 0.f;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) b += __shfl_down_sync(0xffffffffu, b, o);
            if (lane == 0) {
                s_tot = b;
                s_fok = ok ? 1 : 0;
                tm.cs->count += 1u;
            }
        }
    }
    __syncthreads();
    out = s_tot;
    const bool ok = s_fok != 0;
    __syncthreads();
    return ok;
}

// Split-phase FP32 team sum for a one-CTA or cluster team (the small-lattice
// CG overlaps its contractions with the cluster sums).  sum_begin: all
// threads pass their values; the CTA's FP32 sum (fixed order) is pushed to
// every member.  sum_end: all threads; waits for the members and returns
// the total, summed in FP32 in rank order, on every thread.  Nothing but
// __syncthreads-separated work may use the team between the two.
struct SplitSum {
    float w[32];
    float single;
    float tot;
    int ok;
};

__device__ inline void sum_begin(const Team& tm, SplitSum& ss, float x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    if (lane == 0) ss.w[warp] = x;
    __syncthreads();
    if (warp == 0) {
        float a = 0.f;
        if (lane == 0)
            for (int w = 0; w < nw; ++w) a += ss.w[w];
        a = __shfl_sync(0xffffffffu, a, 0);
        if (tm.size == 1) {
            if (lane == 0) ss.single = a;
        } else {
            cluster_push<1, true>(tm, nullptr, a);
        }
    }
}

__device__ inline bool sum_end(const Team& tm, SplitSum& ss, float& out) {
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        if (tm.size == 1) {
            if (lane == 0) {
                ss.tot = ss.single;
                ss.ok = 1;
            }
        } else {
            bool ok = true;
            if (lane == 0) ok = cluster_wait(tm);
            __syncwarp();
            const int par = (int)(tm.cs->count & 1u);
            float b = lane < tm.size ? tm.cs->part_f[par][lane] : 0.f;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) b += __shfl_down_sync(0xffffffffu, b, o);
            __syncwarp();
            if (lane == 0) {
                ss.tot = b;
                ss.ok = ok ? 1 : 0;
                tm.cs->count += 1u;
            }
        }
    }
    __syncthreads();
    out = ss.tot;
    return ss.ok != 0;
}

__device__ __forceinline__ bool finite_d(double a) { return isfinite(a); }

}  // namespace hmc
