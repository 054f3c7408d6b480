// tc_splitk.cuh -- split-K tensor-core applications of M and M^dag with the
// transfer matrix resident in shared memory, for the FP32 iterations of the
// mixed CG on large lattices (operand_mode 5).
//
// GEMM view (site-major, as tc_tile.cuh): D[i][j] = sum_k E'[i][k] B[j][k],
// i = target site (MMA M = 128 per site block), j = 2 tt + {re, im} for the
// tt-th slice of an n-group of ns slices, k = source site.  The team is
// nib x nng thread-block clusters of C CTAs: cluster (ib, ng) owns site block
// ib and n-group ng, and its C CTAs split K into contiguous ranges of
// 16-site steps.  Each CTA loads its rows x K-range of E' once per launch and
// keeps them in shared memory for every application of every solve (E does
// not change), so an application moves only the source vector over the
// CTA's K range, not E.
//
// Split precision with one accumulator (the scaled split of the slice-major
// tile): E' = 2^eE E = E'_hi + E'_lo and s u = B_hi + B_lo, all FP16 with
// plain remainders.  B_lo is stored right after B_hi as further MMA rows,
// so per 16-wide K step two instructions cover the three products:
//     D[:, 0:Nn]   += E'_hi [B_hi; B_lo] (N = 2 Nn) and E'_lo B_hi (N = Nn)
//     D[:, Nn:2Nn]  = E'_hi B_lo
// and the epilogue adds the two column halves.
//
// After the MMAs every CTA stages its partial D as FP32 columns in shared
// memory; after a bounded cluster barrier, CTA rank r of the cluster sums the
// C partials of its share of the n-group's slices through distributed
// shared memory in rank order (deterministic) and runs the fused CG
// epilogue.  Each CTA splits its source with its own power-of-two scale,
// from the largest exponent its source's owners posted, and unscales its
// partial when staging it.  The team's norms travel in the same posted
// words (sequence-numbered slots in global memory) and are summed by every
// CTA in rank order (no atomics; the same bits on every CTA), overlapping
// the next application's copies and MMAs.
//
// The CG iteration uses M^dag's linearity (as the CUDA-core cluster mode):
// with G = E p'_{t+1} carried per target slice, E p' = E r_{t+1} + beta G,
// so M^dag contracts r only, and M contracts u = e^{i phi} q, which the
// M^dag epilogue writes.  Each element (t, i) has one owner CTA for the
// whole solve, which keeps r, p, q, G and the FP32 increment of x of its
// elements in shared memory during a CG segment; r and u also go to global
// memory, where the other CTAs read their K ranges of them.
//
// Shared memory of a CTA (operand area): E'_hi / E'_lo chunks | B chunks
// (the raw FP32 source of chunk j is first copied by cp.async into the
// space of B chunk j, all chunks at once, then split in place) | staging of
// the partial accumulator (in the B area when it fits) | owner vectors.
#pragma once

#include "tc_tile.cuh"

namespace hmc {
namespace tc {

constexpr int kSkMaxChunks = 4;      // K chunks of 64 per CTA (K range <= 256)
static_assert(kSkMaxChunks <= (int)(sizeof(TileBars::skb) / sizeof(uint64_t)),
              "one B barrier per chunk of a standalone application");
constexpr int kSkMaxNn = 128;        // B rows per part (2 x slices of an n-group)
constexpr int kSkMaxCluster = 8;

// Geometry of one CTA of the split-K team.
struct SkGeom {
    int C, ns, Nn, nng, nib;
    int ib, ng, rank;       // site block, n-group, K-range rank (cluster rank)
    int t0, nsl;            // first slice of the n-group, its slices (<= ns)
    int ks0, ks1;           // 16-site K steps [ks0, ks1) of this CTA
    int nch;                // resident chunks of 64 K from 16 * ks0
    int so0, so1;           // owned slices [so0, so1) of the n-group (epilogue)
    uint32_t b_off, s_off;  // B area and staging area (offsets in the operand area)
    uint32_t o_off;         // owner vectors: r, p, q, G, x of the owned elements
    int own;                // owned elements (so1 - so0) * 128
};

__host__ __device__ inline int sk_nn(int ns) { return ((2 * ns + 15) / 16) * 16; }

// Shared-memory bytes of a CTA whose K range spans nch chunks (E' hi/lo,
// the stacked B of every chunk, and the FP32 staging of the partial when it
// does not fit in the B area).
__host__ __device__ inline size_t sk_smem_bytes(int nch, int Nn) {
    const size_t e = (size_t)nch * kAChunkBytes;
    const size_t b = (size_t)nch * 2 * Nn * 128;
    const size_t s = (size_t)Nn * TM * 4;
    return e + (b >= s ? b : b + s);
}
constexpr int kSkOwnerVecs = 5;   // r, p, q, G, x
// ... plus the owner vectors of at most `own_slices` slices.
__host__ __device__ inline size_t sk_smem_total(int nch, int Nn, int own_slices) {
    return sk_smem_bytes(nch, Nn) + (size_t)kSkOwnerVecs * own_slices * TM * 8;
}

// Chunks of 64 K covering at most `steps` 16-site steps from any start.
__host__ __device__ inline int sk_chunks(int steps) { return (steps + 3) / 4; }

__device__ inline SkGeom sk_geom(int team_rank, int C, int ns, int V, int Nt, int Vr, int Vp) {
    SkGeom g;
    g.C = C;
    g.ns = ns;
    g.Nn = sk_nn(ns);
    g.nng = (Nt + ns - 1) / ns;
    g.nib = Vr / TM;
    const int cl = team_rank / C;
    g.rank = team_rank % C;
    g.ib = cl / g.nng;
    g.ng = cl % g.nng;
    g.t0 = g.ng * ns;
    g.nsl = min(ns, Nt - g.t0);
    const int KS = (V + 15) / 16;          // steps holding sites < V
    g.ks0 = KS * g.rank / C;
    g.ks1 = KS * (g.rank + 1) / C;
    g.nch = sk_chunks(g.ks1 - g.ks0);
    g.so0 = g.nsl * g.rank / C;
    g.so1 = g.nsl * (g.rank + 1) / C;
    // The layout follows the largest chunk count of the cluster, not this
    // CTA's own: the members read each other's staged partials at this
    // CTA's offsets (distributed shared memory), so the offsets must agree.
    const int nchx = sk_chunks((KS + C - 1) / C);
    g.b_off = (uint32_t)nchx * kAChunkBytes;
    const uint32_t bbytes = (uint32_t)nchx * 2u * (uint32_t)g.Nn * 128u;
    g.s_off = bbytes >= (uint32_t)g.Nn * TM * 4u ? g.b_off : g.b_off + bbytes;
    g.o_off = (uint32_t)sk_smem_bytes(nchx, g.Nn);
    g.own = (g.so1 - g.so0) * TM;
    (void)Vp;
    return g;
}

// Load this CTA's rows of E' (site block ib) over its K range into the
// chunks of the operand area (TMA, 128-byte swizzle) and wait, bounded.
// All threads call it.
__device__ inline bool sk_load_E(TcState& st, const SkGeom& g, const CUtensorMap* mhi,
                                 const CUtensorMap* mlo) {
    TileBars& b = *st.bars;
    __syncthreads();
    if (threadIdx.x == 0) {
        const uint32_t bar = smem_u32(&b.res_full);
        mbar_arrive_expect_tx(bar, (uint32_t)g.nch * kAChunkBytes);
        for (int j = 0; j < g.nch; ++j) {
            const uint32_t dst = smem_u32(st.base + (size_t)j * kAChunkBytes);
            const int x = 16 * g.ks0 + KCH * j;   // a multiple of 16 elements
            tma_load_2d(dst, mhi, x, g.ib * TM, bar);
            tma_load_2d(dst + kATileBytes, mlo, x, g.ib * TM, bar);
        }
    }
    const bool ok = mbar_wait(smem_u32(&b.res_full), st.nres & 1, st.status);
    st.nres += 1;
    __syncthreads();
    return ok;
}

// Bounded barrier over the CTAs of this cluster (release / acquire at
// cluster scope): the members' shared-memory writes before it are visible
// to every member's reads after it.  All threads.
__device__ inline bool sk_cluster_sync(Team& tcl) {
    asm volatile("fence.acq_rel.cluster;" ::: "memory");
    return team_barrier(tcl);
}

// Team words of the split-K iteration.  After each epilogue every CTA of
// the inner team posts one 64-bit word to its slot [seq & 1][rank]:
//     seq (24 bits) | max exponent (8 bits) | FP32 partial norm (32 bits),
// the max exponent being the biased FP32 exponent of the largest |Re|, |Im|
// of the source elements it has just written.  The post publishes those
// writes (block barrier, fence, then the store), so it doubles as the
// owner's "data ready" flag: a consumer waits only for the owners of its K
// range, takes their largest exponent as its operand scale, and copies.
// The norm is summed later, before the epilogue that needs it, by every
// CTA reading all slots in rank order (no atomics; the same bits on every
// CTA), so the sum overlaps the copies and the MMAs.  Two slot buffers
// suffice: a CTA posts seq + 2 only after reading every slot of seq + 1,
// which every CTA posts only after its own reads of seq are done.
// Each slot has its own 128-byte line (every CTA reads every slot once per
// sum; packed slots put all of those reads on a few lines).
constexpr int kSlotStride = 16;   // 64-bit words
constexpr int kGatherSlots = 2 * kMaxTeam * kSlotStride;
__device__ __forceinline__ size_t sk_slot(unsigned seq, int rank) {
    return ((size_t)(seq & 1u) * kMaxTeam + (size_t)rank) * kSlotStride;
}

__device__ __forceinline__ unsigned long long sk_word(unsigned seq, unsigned mexp, float part) {
    return ((unsigned long long)(seq & 0xffffffu) << 40) |
           ((unsigned long long)(mexp & 0xffu) << 32) | (unsigned long long)__float_as_uint(part);
}
__device__ __forceinline__ bool sk_word_is(unsigned long long w, unsigned seq) {
    return (unsigned)(w >> 40) == (seq & 0xffffffu);
}

// Release store / acquire load of a team word at GPU scope.
__device__ __forceinline__ void st_release_u64(unsigned long long* p, unsigned long long v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// Bounded polling: every 16th probe checks the team status and the time.
__device__ __forceinline__ bool sk_poll_expired(const Team& ti, unsigned k, uint64_t& t0) {
    if ((k & 15u) != 0) return false;
    if (t0 == 0) t0 = global_ns();
    if (team_failed(ti) || global_ns() - t0 > wait_limit_ns(ti.status)) {
        if (!team_failed(ti)) set_status(ti.status, HMC_ERR_TIMEOUT);
        return true;
    }
    return false;
}

// Post (all threads): the block's sum of `part` and max of `mx` under seq.
__device__ inline void sk_post(const Team& ti, unsigned long long* slots, unsigned seq,
                               float part, float mx) {
    __shared__ float s_p[32], s_m[32];
    // this thread's shared-memory writes (split operands, staged partial)
    // before the TMA loads that will overwrite them after the post
    fence_proxy_async();
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        part += __shfl_down_sync(0xffffffffu, part, o);
        mx = fmaxf(mx, __shfl_down_sync(0xffffffffu, mx, o));
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    if (lane == 0) {
        s_p[warp] = part;
        s_m[warp] = mx;
    }
    __syncthreads();   // also: every thread's epilogue writes precede the fence below
    if (threadIdx.x == 0) {
        float a = 0.f, m = 0.f;
        for (int w = 0; w < nw; ++w) {
            a += s_p[w];
            m = fmaxf(m, s_m[w]);
        }
        const unsigned mexp = (__float_as_uint(m) >> 23) & 0xffu;
        // release: the block's writes (ordered before by the barrier above)
        // become visible with the word
        st_release_u64(slots + sk_slot(seq, ti.rank), sk_word(seq, mexp, a));
    }
}

// Team ranks of the CTAs that own the source elements of this CTA's K
// range: the target slices of its n-group shifted to their source slices
// (t + 1 for M^dag, t - 1 for M, cyclic), sites 16 ks0 .. min(16 ks1, V).
// At most (C + 1) ranks per site block and 3 site blocks (K range <= 256
// sites).  The other members of this CTA's cluster come first: they read
// its staged partial through distributed shared memory, so its next source
// may land there only after their posts.  Returns -1 beyond kSkMaxOwners.
constexpr int kSkMaxOwners = 64;
__device__ inline int sk_owner_list(const SkGeom& g, int V, int Nt, bool dag, int* list,
                                    int team_rank) {
    int n = 0;
    const int cl0 = team_rank - g.rank;
    for (int q = 0; q < g.C; ++q)
        if (q != g.rank) list[n++] = cl0 + q;
    const int k0 = 16 * g.ks0, k1 = min(16 * g.ks1, V);
    if (k1 <= k0) return 0;
    const int ib0 = k0 / TM, ib1 = (k1 - 1) / TM;
    for (int tt = 0; tt < g.nsl; ++tt) {
        int ts = g.t0 + tt + (dag ? 1 : -1);
        ts = ts < 0 ? Nt - 1 : (ts >= Nt ? 0 : ts);
        const int ngo = ts / g.ns, t0o = ngo * g.ns, nslo = min(g.ns, Nt - t0o), rr = ts - t0o;
        int ro = 0;   // the owner: the last rank whose first owned slice is <= rr
        while (ro + 1 < g.C && nslo * (ro + 1) / g.C <= rr) ++ro;
        for (int ib = ib0; ib <= ib1; ++ib) {
            const int rank = (ib * g.nng + ngo) * g.C + ro;
            bool seen = false;
            for (int q = 0; q < n; ++q) seen |= list[q] == rank;
            if (seen) continue;
            if (n == kSkMaxOwners) return -1;
            list[n++] = rank;
        }
    }
    return n;
}

// Warp 0: wait (bounded) until the n ranks in `list` have posted seq and
// return the largest max exponent among them; each lane reads its owner's
// word with acquire semantics, and the block barrier that the caller runs
// next orders the other threads after those reads.
// `mexp` starts from `own_mexp` (0 when the list covers every owner).
__device__ inline bool sk_wait_owners(const Team& ti, const unsigned long long* slots,
                                      unsigned seq, const int* list, int n, unsigned own_mexp,
                                      unsigned& mexp) {
    const int lane = threadIdx.x & 31;
    bool ok = true;
    unsigned m = own_mexp;
    for (int q = lane; q < n && ok; q += 32) {
        const unsigned long long* p = slots + sk_slot(seq, list[q]);
        unsigned long long w = ld_acquire_u64(p);
        uint64_t t0 = 0;
        for (unsigned k = 1; !sk_word_is(w, seq); ++k) {
            if (sk_poll_expired(ti, k, t0)) { ok = false; break; }
            __nanosleep(32);
            w = ld_acquire_u64(p);
        }
        m = max(m, (unsigned)(w >> 32) & 0xffu);
    }
    ok = __all_sync(0xffffffffu, ok);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    mexp = m;
    return ok;
}

// Warp 0: the sum of the partial norms of all team slots posted under seq,
// in a fixed order (lane l adds ranks l, l + 32, ...; then a fixed shuffle
// tree), so every CTA gets the same bits; also the largest max exponent
// of the team (gmexp).  sk_sum_begin loads the first
// kSumPre slots of each lane (their loads in flight while the caller does
// other work); sk_sum_end polls those not yet posted, adds the rest of the
// team and returns the sum on every lane.
constexpr int kSumPre = 4;
struct SkSum {
    unsigned long long w[kSumPre];
};
__device__ __forceinline__ void sk_sum_begin(const Team& ti, const unsigned long long* slots,
                                             unsigned seq, SkSum& ss) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int b = 0; b < kSumPre; ++b) {
        const int r = lane + 32 * b;
        ss.w[b] = r < ti.size ? *(const volatile unsigned long long*)(slots + sk_slot(seq, r))
                              : sk_word(seq, 0u, 0.f);
    }
}
__device__ inline bool sk_sum_end(const Team& ti, const unsigned long long* slots, unsigned seq,
                                  SkSum& ss, float& out, unsigned& gmexp) {
    const int lane = threadIdx.x & 31;
    bool ok = true;
    float acc = 0.f;
    unsigned gm = 0;
    for (int r = lane, b = 0; r < ti.size && ok; r += 32, ++b) {
        unsigned long long w =
            b < kSumPre ? ss.w[b] : *(const volatile unsigned long long*)(slots + sk_slot(seq, r));
        uint64_t t0 = 0;
        for (unsigned k = 1; !sk_word_is(w, seq); ++k) {
            if (sk_poll_expired(ti, k, t0)) { ok = false; break; }
            __nanosleep(64);
            w = *(const volatile unsigned long long*)(slots + sk_slot(seq, r));
        }
        acc += __uint_as_float((unsigned)(w & 0xffffffffull));
        gm = max(gm, (unsigned)(w >> 32) & 0xffu);
    }
    ok = __all_sync(0xffffffffu, ok);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        acc += __shfl_down_sync(0xffffffffu, acc, o);
        gm = max(gm, __shfl_xor_sync(0xffffffffu, gm, o));
    }
    out = __shfl_sync(0xffffffffu, acc, 0);
    gmexp = gm;
    return ok;
}

// Operand scale 2^e of a source whose largest component has biased
// exponent mexp: largest |component| 2^e in [2^14, 2^15) (e = 0 for zero or
// non-finite sources).
__device__ __forceinline__ void sk_scale(unsigned mexp, float& scale, float& inv) {
    int e = 0;
    if (mexp != 0u && mexp != 0xffu) e = max(-120, min(120, 14 - ((int)mexp - 127)));
    scale = __int_as_float((127 + e) << 23);
    inv = __int_as_float((127 - e) << 23);
}

// B items (slice tt, 8-site group) per thread and chunk: a chunk has
// nsl * 8 <= 512 items, so at most two per thread.
constexpr int kSkItems = 2;

// Thread 0: the MMAs of chunk j (the CTA's K steps 4j .. 4j+3 within its
// range); the last chunk commits the accumulator barrier.
__device__ __forceinline__ void sk_issue_chunk(const TcState& st, const SkGeom& g, int j,
                                               uint32_t bchunk, uint32_t tmem) {
    fence_after_sync();
    const int Nn = g.Nn, nsteps = g.ks1 - g.ks0;
    const uint32_t idesc2 = idesc_f16(TM, 2 * Nn), idesc1 = idesc_f16(TM, Nn);
    const uint32_t ah = smem_u32(st.base + (size_t)j * kAChunkBytes);
    const uint32_t al = ah + kATileBytes;
    for (int kk = 0; kk < 4; ++kk) {
        const int s = 4 * j + kk;
        if (s >= nsteps) break;
        const uint32_t off = (uint32_t)kk * 32u;
        mma_f16(tmem, desc_sw128(ah + off), desc_sw128(bchunk + off), idesc2, s > 0 ? 1u : 0u);
        mma_f16(tmem, desc_sw128(al + off), desc_sw128(bchunk + off), idesc1, 1u);
    }
    if (j == g.nch - 1) mma_commit(smem_u32(&st.bars->acc_full));
}

// Split-K CG source by TMA (thread 0): for every chunk j of this CTA's K
// range, the box of 64 sites from 16 ks0 + 64 j and ns rows from row0 of
// the halo layout (zeros past V and past the last row) into the space of
// B chunk j, completing barrier skb[j].
__device__ __forceinline__ void sk_issue_source(const TcState& st, const SkGeom& g,
                                                const CUtensorMap* map, int row0) {
    if (threadIdx.x != 0) return;
    fence_proxy_async();
    // the owners' generic writes (acquired through their words) before this
    // thread's async-proxy reads of them
    asm volatile("fence.proxy.async.global;" ::: "memory");
    const uint32_t cb = 2u * (uint32_t)g.Nn * 128u;
    const uint32_t bytes = (uint32_t)KCH * (uint32_t)g.ns * 8u;
    for (int j = 0; j < g.nch; ++j) {
        const uint32_t bar = smem_u32(&st.bars->skb[j]);
        mbar_arrive_expect_tx(bar, bytes);
        tma_load_2d(smem_u32(st.base + g.b_off + (size_t)j * cb), map, 16 * g.ks0 + KCH * j,
                    row0, bar);
    }
}

// Split two scaled FP32 values into FP16 pairs hi, lo with x = hi + lo:
// Veltkamp's splitting with the constant 2^13 + 1 leaves hi with 11
// significant bits (exact in FP16 for |x| < 2^16 down to the FP16 normal
// range) and lo = x - hi exact in FP32, then rounded to FP16.  The products
// are kept apart from the sums (no fused multiply-add may merge them).
__device__ __forceinline__ void split_pair_v(float a, float b, uint32_t& hi, uint32_t& lo) {
    const float ta = __fmul_rn(a, 8193.f), tb = __fmul_rn(b, 8193.f);
    const float ha = __fsub_rn(ta, __fsub_rn(ta, a)), hb = __fsub_rn(tb, __fsub_rn(tb, b));
    const __half2 h = __floats2half2_rn(ha, hb);
    const __half2 l = __floats2half2_rn(__fsub_rn(a, ha), __fsub_rn(b, hb));
    hi = *reinterpret_cast<const uint32_t*>(&h);
    lo = *reinterpret_cast<const uint32_t*>(&l);
}

// All threads: chunk by chunk, wait for its source, split it in place with
// `scale` and issue its MMAs (thread 0).  Item (slice tt, 8-site group grp)
// is 64 bytes of raw row tt; its lane reads the four 16-byte pieces starting
// at piece (grp >> 1) & 3 (the eight lanes of a quarter warp then hit eight
// different bank groups) and writes each piece's two sites as four 32-bit
// words (hi/lo x re/im) into the swizzled B rows (conflict-free as well).
// False if a wait failed (status set; every thread returns together).
__device__ __forceinline__ bool sk_convert_and_issue(TcState& st, const SkGeom& g, float scale,
                                                     uint32_t tmem) {
    const int Nn = g.Nn;
    const uint32_t cb = 2u * (uint32_t)Nn * 128u;
    const int per_chunk = g.nsl * 8;
    const int kend = 16 * g.ks1;
    const uint32_t phase = st.nskb & 1u;
    st.nskb += 1;
    for (int j = 0; j < g.nch; ++j) {
        uint8_t* ch = st.base + g.b_off + (size_t)j * cb;
        bool ok = mbar_wait(smem_u32(&st.bars->skb[j]), phase, st.status);
        if (!__syncthreads_and(ok)) {
            // MMAs of earlier chunks are in flight: commit them, so the
            // teardown waits for them before it frees the accumulator
            if (j > 0) {
                if (threadIdx.x == 0) mma_commit(smem_u32(&st.bars->acc_full));
                st.ntile += 1;
            }
            return false;
        }
        float4 v[kSkItems][4];
        const float4* raw = reinterpret_cast<const float4*>(ch);
#pragma unroll
        for (int m = 0; m < kSkItems; ++m) {
            const int r = threadIdx.x + m * NTHR;
            if (r < per_chunk) {
                const int tt = r >> 3, grp = r & 7, rot = (grp >> 1) & 3;
#pragma unroll
                for (int e = 0; e < 4; ++e) v[m][e] = raw[tt * 32 + grp * 4 + ((e + rot) & 3)];
            }
        }
        __syncthreads();   // every read of the raw chunk before the split overwrites it
#pragma unroll
        for (int m = 0; m < kSkItems; ++m) {
            const int r = threadIdx.x + m * NTHR;
            const int tt = r >> 3, grp = r & 7, rot = (grp >> 1) & 3;
            const int kb = 16 * g.ks0 + KCH * j + 8 * grp;
            if (r < per_chunk && kb < kend) {
                const int jr = 2 * tt, ji = jr + 1;
                uint8_t* hr = ch + jr * 128 + ((grp ^ (jr & 7)) << 4);
                uint8_t* hm = ch + ji * 128 + ((grp ^ (ji & 7)) << 4);
                uint8_t* lr = hr + (size_t)Nn * 128;
                uint8_t* lm = hm + (size_t)Nn * 128;
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int pc = ((e + rot) & 3) * 4;
                    const float4 a = v[m][e];
                    uint32_t h0, l0, h1, l1;
                    split_pair_v(a.x * scale, a.z * scale, h0, l0);   // re of sites 2pc', +1
                    split_pair_v(a.y * scale, a.w * scale, h1, l1);   // im
                    *reinterpret_cast<uint32_t*>(hr + pc) = h0;
                    *reinterpret_cast<uint32_t*>(lr + pc) = l0;
                    *reinterpret_cast<uint32_t*>(hm + pc) = h1;
                    *reinterpret_cast<uint32_t*>(lm + pc) = l1;
                }
            }
        }
        fence_proxy_async();
        __syncthreads();
        if (threadIdx.x == 0) sk_issue_chunk(st, g, j, smem_u32(ch), tmem);
    }
    return true;
}

// Sites i .. i+3 of halo row h of a source, split: FP16 hi and lo of the
// values times sc (zeros for sites >= V) into rows 2h (Re) and 2h + 1 (Im)
// of the hi and lo planes (row stride Vp; 8-byte stores).
__device__ __forceinline__ void sk_store_b16(__half_raw* bh, __half_raw* bl, int Vp, int V, int h,
                                             int i, const float2 (&v)[4], float sc) {
    float re[4], im[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        re[e] = i + e < V ? v[e].x * sc : 0.f;
        im[e] = i + e < V ? v[e].y * sc : 0.f;
    }
    uint32_t h0, l0, h1, l1, h2, l2, h3, l3;
    split_pair_v(re[0], re[1], h0, l0);
    split_pair_v(re[2], re[3], h1, l1);
    split_pair_v(im[0], im[1], h2, l2);
    split_pair_v(im[2], im[3], h3, l3);
    const size_t ore = (size_t)(2 * h) * Vp + i, oim = ore + Vp;
    *reinterpret_cast<uint2*>(bh + ore) = make_uint2(h0, h1);
    *reinterpret_cast<uint2*>(bl + ore) = make_uint2(l0, l1);
    *reinterpret_cast<uint2*>(bh + oim) = make_uint2(h2, h3);
    *reinterpret_cast<uint2*>(bl + oim) = make_uint2(l2, l3);
}

// Split-K CG source already split by its owners (thread 0 only): for every
// chunk j, the FP16 hi and lo boxes (64 sites from 16 ks0 + 64 j, sk_nn(ns)
// rows from row16) straight into the swizzled B layout of chunk j, one
// barrier per chunk; then chunk by chunk wait and issue the MMAs.  On a
// failed wait the accumulator barrier is committed all the same (the
// caller's wait for it then returns) and the status is set.
__device__ __forceinline__ void sk_issue_b16(TcState& st, const SkGeom& g, const CUtensorMap* mhi,
                                             const CUtensorMap* mlo, int row16, uint32_t tmem) {
    const uint32_t phase = st.nskb & 1u;
    st.nskb += 1;
    if (threadIdx.x != 0) return;
    asm volatile("fence.proxy.async.global;" ::: "memory");   // as sk_issue_source
    const uint32_t cb = 2u * (uint32_t)g.Nn * 128u;
    for (int j = 0; j < g.nch; ++j) {
        const uint32_t bar = smem_u32(&st.bars->skb[j]);
        const uint32_t dst = smem_u32(st.base + g.b_off + (size_t)j * cb);
        const int x = 16 * g.ks0 + KCH * j;
        mbar_arrive_expect_tx(bar, cb);
        tma_load_2d(dst, mhi, x, row16, bar);
        tma_load_2d(dst + (uint32_t)g.Nn * 128u, mlo, x, row16, bar);
    }
    for (int j = 0; j < g.nch; ++j) {
        if (!mbar_wait(smem_u32(&st.bars->skb[j]), phase, st.status)) {
            mma_commit(smem_u32(&st.bars->acc_full));
            return;
        }
        sk_issue_chunk(st, g, j, smem_u32(st.base + g.b_off + (size_t)j * cb), tmem);
    }
}

// After the MMAs are issued: wait for the accumulator and stage it in
// shared memory as FP32 columns [column][128 rows], multiplied by
// stage_scale (the inverse of this CTA's operand scale, exact: a power of
// two), or, with col_inv, by the inverse scale of the column's slice and
// this CTA's K range, col_inv[(t0 + column / 2) * C + rank] (standalone
// applications).  All threads; false if the wait failed (status set).
__device__ __forceinline__ bool sk_stage(TcState& st, const SkGeom& g, float stage_scale,
                                         const float* col_inv = nullptr, int Nt = 0) {
    TileBars& bars = *st.bars;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t tmem = bars.tmem_base;
    const int Nn = g.Nn;
    bool ok = mbar_wait(smem_u32(&bars.acc_full), st.ntile & 1, st.status);
    st.ntile += 1;
    fence_after_sync();
    ok = __all_sync(0xffffffffu, ok);
    float* stg = reinterpret_cast<float*>(st.base + g.s_off);
    if (ok) {
        // the two warps of a TMEM lane quarter split the 16-column blocks
        const int nb = Nn / 16, half = (nb + 1) / 2;
        const bool first = warp >= 4;
        const int b0 = first ? 0 : half, b1 = first ? half : nb;
        const int row = (warp & 3) * 32 + lane;
        const uint32_t tl = tmem + ((uint32_t)((warp & 3) * 32) << 16);
        for (int cb = b0; cb < b1; ++cb) {
            float m[16], l[16];
            tmem_ld16(tl + (uint32_t)(cb * 16), m);
            tmem_ld16(tl + (uint32_t)(Nn + cb * 16), l);
#pragma unroll
            for (int e = 0; e < 16; ++e) {
                float sc = stage_scale;
                if (col_inv) {
                    const int t = g.t0 + ((cb * 16 + e) >> 1);
                    sc = t < Nt ? col_inv[t * g.C + g.rank] : 0.f;
                }
                stg[(cb * 16 + e) * TM + row] = (m[e] + l[e]) * sc;
            }
        }
    }
    fence_before_sync();
    __syncthreads();
    return ok;
}

// After sk_stage: sync the cluster (HW: the hardware cluster barrier of a
// standalone launch, which every thread reaches; else the bounded barrier
// of the CG team), then this CTA's owned outputs: the C partials summed in
// rank order through distributed shared memory and multiplied by unscale,
// then epi.store(t, i, owner index, w[4]).
template <bool HW, class Epi>
__device__ __forceinline__ bool sk_reduce(const TcState& st, const SkGeom& g, Team& tcl, int V,
                                          float unscale, Epi& epi) {
    if constexpr (HW) {
        cluster_barrier_all();   // every member's partial staged (release / acquire)
    } else {
        if (!sk_cluster_sync(tcl)) return false;
    }
    const float* stg = reinterpret_cast<const float*>(st.base + g.s_off);
    // owned slices: sum the C partials in rank order, then the epilogue
    const uint32_t stg_s = smem_u32(stg);
    const int items = (g.so1 - g.so0) * (TM / 4);
    for (int w = threadIdx.x; w < items; w += blockDim.x) {
        const int tl = w / (TM / 4);
        const int tt = g.so0 + tl;
        const int i4 = (w % (TM / 4)) * 4;
        const int i = g.ib * TM + i4;
        if (i >= V) continue;
        const uint32_t ore = stg_s + (uint32_t)(((2 * tt) * TM + i4) * 4);
        const uint32_t oim = ore + (uint32_t)(TM * 4);
        epi.prefetch(g.t0 + tt, i);
        // the members' partials in two groups of four loads in flight, added
        // in rank order
        float4 sr = make_float4(0.f, 0.f, 0.f, 0.f), si = sr;
#pragma unroll
        for (int q0 = 0; q0 < kSkMaxCluster; q0 += 4) {
            float4 xr[4], xi[4];
#pragma unroll
            for (int d = 0; d < 4; ++d) {
                const int q = q0 + d;
                if (q < g.C) {
                    uint32_t ar, ai;
                    asm("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ar) : "r"(ore), "r"(q));
                    asm("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ai) : "r"(oim), "r"(q));
                    asm("ld.shared::cluster.v4.f32 {%0, %1, %2, %3}, [%4];"
                        : "=f"(xr[d].x), "=f"(xr[d].y), "=f"(xr[d].z), "=f"(xr[d].w)
                        : "r"(ar)
                        : "memory");
                    asm("ld.shared::cluster.v4.f32 {%0, %1, %2, %3}, [%4];"
                        : "=f"(xi[d].x), "=f"(xi[d].y), "=f"(xi[d].z), "=f"(xi[d].w)
                        : "r"(ai)
                        : "memory");
                }
            }
#pragma unroll
            for (int d = 0; d < 4; ++d) {
                if (q0 + d < g.C) {
                    sr.x += xr[d].x; sr.y += xr[d].y; sr.z += xr[d].z; sr.w += xr[d].w;
                    si.x += xi[d].x; si.y += xi[d].y; si.z += xi[d].z; si.w += xi[d].w;
                }
            }
        }
        const float2 wv[4] = {make_float2(sr.x * unscale, si.x * unscale),
                              make_float2(sr.y * unscale, si.y * unscale),
                              make_float2(sr.z * unscale, si.z * unscale),
                              make_float2(sr.w * unscale, si.w * unscale)};
        epi.store(g.t0 + tt, i, tl * TM + i4, wv);
    }
    return true;
}

template <bool HW, class Epi>
__device__ __forceinline__ bool sk_finish(TcState& st, const SkGeom& g, Team& tcl, int V,
                                          float unscale, Epi& epi, const float* col_inv = nullptr,
                                          int Nt = 0) {
    const bool ok = sk_stage(st, g, 1.f, col_inv, Nt);
    if constexpr (HW) {
        // every thread reaches the hardware cluster barrier, failed or not
        const bool r = sk_reduce<true>(st, g, tcl, V, unscale, epi);
        return ok && r;
    } else {
        if (!ok) return false;
        return sk_reduce<false>(st, g, tcl, V, unscale, epi);
    }
}

// Four sites i .. i+3 of row `row` of a [rows][V] FP32 complex array
// (16-byte stores when all four are in range).
__device__ __forceinline__ void sk_store_halo(float2* a, int V, int row, int i,
                                              const float2 (&v)[4]) {
    float2* p = a + (size_t)row * V + i;
    if (i + 4 <= V) {
        *reinterpret_cast<float4*>(p) = make_float4(v[0].x, v[0].y, v[1].x, v[1].y);
        *reinterpret_cast<float4*>(p + 2) = make_float4(v[2].x, v[2].y, v[3].x, v[3].y);
    } else {
#pragma unroll
        for (int e = 0; e < 4; ++e)
            if (i + e < V) p[e] = v[e];
    }
}

// Owner vectors of a CTA in shared memory: FP32 complex arrays of g.own
// elements, owner index (slice - so0) * 128 + (site - 128 ib).
struct SkOwner {
    float2 *r, *p, *q, *G, *x;
    __device__ __forceinline__ void init(uint8_t* base, const SkGeom& g) {
        float2* o = reinterpret_cast<float2*>(base + g.o_off);
        r = o;
        p = o + g.own;
        q = o + 2 * g.own;
        G = o + 3 * g.own;
        x = o + 4 * g.own;
    }
};

// Owner elements of a CTA: (global offset, owner index) for each valid one.
#define HMC_SK_OWNED(o, oi, g, c)                                                       \
    for (int oi = threadIdx.x; oi < (g).own; oi += blockDim.x)                          \
        if ((g).ib * TM + (oi % TM) < (c).V)                                            \
            for (size_t o = (size_t)((g).t0 + (g).so0 + oi / TM) * (c).V +              \
                            (g).ib * TM + (oi % TM), _once = 0;                         \
                 _once == 0; _once = 1)

// M^dag epilogue of the split-K CG iteration at (t, i .. i+3): with
// w = E r_{t+1},  G = w + beta G,  p' = r + beta p,
// q = p' - g s_{t+1} e^{-i phi_t} G,  u = e^{i phi_t} q (g = hop: 1 for M,
// the hop factor of the heavy operator M_g).  Updates G, p (= p'),
// q in shared memory and writes u to global memory; sums |q|^2.
struct SkEpiDag {
    SkOwner ow;
    float2* u;       // halo rows [Nt + 2][V]
    __half_raw *bh, *bl;   // FP16 split planes of u (null: not written)
    float bscale;
    int Vp;
    const float2* cis;
    float beta;
    float hop;       // g of the operator 1 - g S E D (1 for M itself)
    int V, Nt;
    float acc;       // |q|^2 of the owned elements
    float mx;        // largest |Re|, |Im| of the u written
    float4 c0, c1;   // prefetched phases
    __device__ __forceinline__ void prefetch(int t, int i) {
        const size_t o = (size_t)t * V + i;
        if (i + 4 <= V) {
            c0 = *reinterpret_cast<const float4*>(cis + o);
            c1 = *reinterpret_cast<const float4*>(cis + o + 2);
        } else {
            const float2 a = cis[o], b = i + 1 < V ? cis[o + 1] : make_float2(1.f, 0.f);
            const float2 d = i + 2 < V ? cis[o + 2] : make_float2(1.f, 0.f);
            const float2 e = i + 3 < V ? cis[o + 3] : make_float2(1.f, 0.f);
            c0 = make_float4(a.x, a.y, b.x, b.y);
            c1 = make_float4(d.x, d.y, e.x, e.y);
        }
    }
    __device__ __forceinline__ void store(int t, int i, int oi, const float2 (&w)[4]) {
        const float sg = (t == Nt - 1) ? -1.f : 1.f;
        const float2 ph[4] = {make_float2(c0.x, c0.y), make_float2(c0.z, c0.w),
                              make_float2(c1.x, c1.y), make_float2(c1.z, c1.w)};
        float2 us[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const float2 rv = ow.r[oi + e], g0 = ow.G[oi + e], p0 = ow.p[oi + e];
            const float2 gv = make_float2(fmaf(beta, g0.x, w[e].x), fmaf(beta, g0.y, w[e].y));
            const float2 pv = make_float2(fmaf(beta, p0.x, rv.x), fmaf(beta, p0.y, rv.y));
            const float2 cg = cmulcf(ph[e], gv);
            const float sh = sg * hop;
            const float2 qv = make_float2(pv.x - sh * cg.x, pv.y - sh * cg.y);
            ow.G[oi + e] = gv;
            ow.p[oi + e] = pv;
            ow.q[oi + e] = qv;
            us[e] = cmulf(ph[e], qv);
            if (i + e < V) {
                acc = fmaf(qv.x, qv.x, fmaf(qv.y, qv.y, acc));
                mx = fmaxf(mx, fmaxf(fabsf(us[e].x), fabsf(us[e].y)));
            }
        }
        // halo layout: row t + 1; slice Nt - 1 also in row 0 (M's source of slice 0)
        sk_store_halo(u, V, t + 1, i, us);
        if (t == Nt - 1) sk_store_halo(u, V, 0, i, us);
        if (bh) {
            sk_store_b16(bh, bl, Vp, V, t + 1, i, us, bscale);
            if (t == Nt - 1) sk_store_b16(bh, bl, Vp, V, 0, i, us, bscale);
        }
    }
};

// M epilogue of the split-K CG iteration at (t, i .. i+3): with
// w = E u_{t-1},  Mq = q - g s_t w,  x += alpha p,  r -= alpha Mq.  Updates x
// and r in shared memory, writes r to global memory; sums |r|^2.
struct SkEpiM {
    SkOwner ow;
    float2* r;       // halo rows [Nt + 2][V]
    __half_raw *bh, *bl;   // FP16 split planes of r (null: not written)
    float bscale;
    int Vp;
    float alpha;
    float hop;       // g of the operator 1 - g S E D (1 for M itself)
    int V, Nt;
    float acc;       // |r|^2 of the owned elements
    float mx;        // largest |Re|, |Im| of the r written
    __device__ __forceinline__ void prefetch(int, int) {}
    __device__ __forceinline__ void store(int t, int i, int oi, const float2 (&w)[4]) {
        const float sg = (t == 0) ? -hop : hop;
        float2 rs[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const float2 qv = ow.q[oi + e], pv = ow.p[oi + e];
            float2 xv = ow.x[oi + e], rv = ow.r[oi + e];
            const float2 mq = make_float2(qv.x - sg * w[e].x, qv.y - sg * w[e].y);
            xv.x = fmaf(alpha, pv.x, xv.x);
            xv.y = fmaf(alpha, pv.y, xv.y);
            rv.x = fmaf(-alpha, mq.x, rv.x);
            rv.y = fmaf(-alpha, mq.y, rv.y);
            ow.x[oi + e] = xv;
            ow.r[oi + e] = rv;
            rs[e] = rv;
            if (i + e < V) {
                acc = fmaf(rv.x, rv.x, fmaf(rv.y, rv.y, acc));
                mx = fmaxf(mx, fmaxf(fabsf(rv.x), fabsf(rv.y)));
            }
        }
        // halo layout: row t + 1; slice 0 also in row Nt + 1 (M^dag's source of slice Nt - 1)
        sk_store_halo(r, V, t + 1, i, rs);
        if (t == 0) sk_store_halo(r, V, Nt + 1, i, rs);
        if (bh) {
            sk_store_b16(bh, bl, Vp, V, t + 1, i, rs, bscale);
            if (t == 0) sk_store_b16(bh, bl, Vp, V, Nt + 1, i, rs, bscale);
        }
    }
};

// Epilogue of a standalone application at (t, i .. i+3): with
// w = (E u)_t (the staged partials already unscaled by their operand
// scales; the sum times 2^-eE),
//     M:      out_t = in_t - s_t w                      (s_0 = -1)
//     M^dag:  out_t = in_t - s_{t+1} e^{-i phi_t} w     (s_Nt = -1)
template <bool DAG>
struct SkEpiOut {
    const float2* in;
    float2* out;
    const float2* cis;   // FP32 e^{i phi} (M^dag)
    int V, Nt;
    float4 c0, c1;
    __device__ __forceinline__ void prefetch(int t, int i) {
        if (!DAG) return;
        const size_t o = (size_t)t * V + i;
        if (i + 4 <= V) {
            c0 = *reinterpret_cast<const float4*>(cis + o);
            c1 = *reinterpret_cast<const float4*>(cis + o + 2);
        } else {
            const float2 a = cis[o], b = i + 1 < V ? cis[o + 1] : make_float2(1.f, 0.f);
            const float2 d = i + 2 < V ? cis[o + 2] : make_float2(1.f, 0.f);
            const float2 e = i + 3 < V ? cis[o + 3] : make_float2(1.f, 0.f);
            c0 = make_float4(a.x, a.y, b.x, b.y);
            c1 = make_float4(d.x, d.y, e.x, e.y);
        }
    }
    __device__ __forceinline__ void store(int t, int i, int, const float2 (&w)[4]) {
        const size_t o = (size_t)t * V + i;
        const float sg = DAG ? ((t == Nt - 1) ? -1.f : 1.f) : ((t == 0) ? -1.f : 1.f);
        const float2 ph[4] = {make_float2(c0.x, c0.y), make_float2(c0.z, c0.w),
                              make_float2(c1.x, c1.y), make_float2(c1.z, c1.w)};
        float2 a[4];
        if (i + 4 <= V) {
            const float4 a0 = *reinterpret_cast<const float4*>(in + o);
            const float4 a1 = *reinterpret_cast<const float4*>(in + o + 2);
            a[0] = make_float2(a0.x, a0.y);
            a[1] = make_float2(a0.z, a0.w);
            a[2] = make_float2(a1.x, a1.y);
            a[3] = make_float2(a1.z, a1.w);
        } else {
#pragma unroll
            for (int e = 0; e < 4; ++e) a[e] = i + e < V ? in[o + e] : make_float2(0.f, 0.f);
        }
        float2 r[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            float2 wv = w[e];
            if (DAG) wv = cmulcf(ph[e], wv);
            r[e] = make_float2(a[e].x - sg * wv.x, a[e].y - sg * wv.y);
        }
        if (i + 4 <= V) {
            *reinterpret_cast<float4*>(out + o) = make_float4(r[0].x, r[0].y, r[1].x, r[1].y);
            *reinterpret_cast<float4*>(out + o + 2) = make_float4(r[2].x, r[2].y, r[3].x, r[3].y);
        } else {
#pragma unroll
            for (int e = 0; e < 4; ++e)
                if (i + e < V) out[o + e] = r[e];
        }
    }
};

}  // namespace tc
}  // namespace hmc
