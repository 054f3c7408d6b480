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
// epilogue.  The team's norms are summed by gather_sum_f: every CTA posts
// its FP32 partial with a sequence number to a slot in global memory and
// every CTA adds all slots in rank order (no atomics; the same bits on every
// CTA).
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
    g.b_off = (uint32_t)g.nch * kAChunkBytes;
    const uint32_t bbytes = (uint32_t)g.nch * 2u * (uint32_t)g.Nn * 128u;
    g.s_off = bbytes >= (uint32_t)g.Nn * TM * 4u ? g.b_off : g.b_off + bbytes;
    g.o_off = (uint32_t)sk_smem_bytes(g.nch, g.Nn);
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

// Source of the B operand: FP32 vector, or (refresh) the FP64 residual.
struct SkSrc {
    const float2* f;
    const double2* d;
    bool use_d;
    int V;
    __device__ __forceinline__ float2 one(size_t o) const {
        if (use_d) {
            const double2 a = d[o];
            return make_float2((float)a.x, (float)a.y);
        }
        return f[o];
    }
    __device__ __forceinline__ void load8(int ts, int kb, float2 (&v)[8]) const {
        const size_t o = (size_t)ts * V + kb;
        if (use_d || kb + 8 > V) {
#pragma unroll
            for (int e = 0; e < 8; ++e)
                v[e] = kb + e < V ? one(o + e) : make_float2(0.f, 0.f);
            return;
        }
        const float4* s4 = reinterpret_cast<const float4*>(f + o);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const float4 a = s4[e];
            v[2 * e] = make_float2(a.x, a.y);
            v[2 * e + 1] = make_float2(a.z, a.w);
        }
    }
};

// FP16 split with a plain remainder, 8 values packed per uint4.
__device__ __forceinline__ void split8_plain(const float (&x)[8], uint4& hi, uint4& lo) {
    uint32_t h[4], l[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const __half h0 = __float2half_rn(x[2 * e]);
        const __half h1 = __float2half_rn(x[2 * e + 1]);
        const __half l0 = __float2half_rn(x[2 * e] - __half2float(h0));
        const __half l1 = __float2half_rn(x[2 * e + 1] - __half2float(h1));
        h[e] = (uint32_t)__half_as_ushort(h0) | ((uint32_t)__half_as_ushort(h1) << 16);
        l[e] = (uint32_t)__half_as_ushort(l0) | ((uint32_t)__half_as_ushort(l1) << 16);
    }
    hi = make_uint4(h[0], h[1], h[2], h[3]);
    lo = make_uint4(l[0], l[1], l[2], l[3]);
}

// Bounded barrier over the CTAs of this cluster (release / acquire at
// cluster scope): the members' shared-memory writes before it are visible
// to every member's reads after it.  All threads.
__device__ inline bool sk_cluster_sync(Team& tcl) {
    asm volatile("fence.acq_rel.cluster;" ::: "memory");
    return team_barrier(tcl);
}

// Team sum of one FP32 value per thread over the inner team without
// atomics.  Every CTA posts its fixed-order sum with the sequence number
// seq to slot [seq & 1][rank]; CTA 0 waits (bounded) until every slot of
// that buffer carries seq, adds them in rank order and posts the total with
// seq to the result word [seq & 1]; every CTA waits (bounded) for that word.
// Two buffers suffice: a CTA posts sync seq + 2 only after reading the
// result of seq + 1, which CTA 0 writes only after every CTA has posted
// seq + 1, each of them after reading the result of seq.  One CTA polling
// all slots and the others one word each keeps the polling traffic on the
// few L2 lines involved small (every CTA polling every slot saturated them
// and slowed all other memory traffic).  Each post and the result publish
// the poster's global writes before it (fence, then store).  Result on
// every thread.
constexpr int kPollBatch = 8;
constexpr int kGatherSlots = 2 * kMaxTeam + 32;   // two slot buffers, two result lines
__device__ inline bool gather_sum_f(const Team& ti, unsigned long long* slots, unsigned& seq,
                                    float x, float& out) {
    __shared__ float s_w[32];
    __shared__ float s_tot;
    __shared__ int s_ok;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    if (lane == 0) s_w[warp] = x;
    seq += 1u;
    __syncthreads();
    unsigned long long* buf = slots + (size_t)(seq & 1u) * kMaxTeam;
    unsigned long long* res = slots + 2 * kMaxTeam + 16 * (seq & 1u);   // own 128-byte line
    const unsigned long long tag = (unsigned long long)seq << 32;
    if (warp == 0) {
        if (lane == 0) {
            float a = 0.f;
            for (int w = 0; w < nw; ++w) a += s_w[w];
            __threadfence();
            *reinterpret_cast<volatile unsigned long long*>(buf + ti.rank) =
                tag | (unsigned long long)__float_as_uint(a);
        }
        __syncwarp();
        bool ok = true;
        uint64_t t0 = 0;
        auto timed_out = [&](unsigned n) {
            if ((n & 15u) != 0) return false;
            if (t0 == 0) t0 = global_ns();
            if (team_failed(ti) || global_ns() - t0 > wait_limit_ns(ti.status)) {
                if (!team_failed(ti)) set_status(ti.status, HMC_ERR_TIMEOUT);
                return true;
            }
            return false;
        };
        if (ti.rank == 0) {
            const volatile unsigned long long* vb = buf;
            float acc = 0.f;
            for (int base = lane; base < ti.size && ok; base += 32 * kPollBatch) {
                unsigned long long v[kPollBatch];
#pragma unroll
                for (int b = 0; b < kPollBatch; ++b) {
                    const int r = base + 32 * b;
                    v[b] = r < ti.size ? vb[r] : tag;
                }
                for (unsigned n = 1;; ++n) {
                    bool all = true;
#pragma unroll
                    for (int b = 0; b < kPollBatch; ++b) all &= (v[b] >> 32) == (tag >> 32);
                    if (all) break;
                    if (timed_out(n)) { ok = false; break; }
                    __nanosleep(32);
#pragma unroll
                    for (int b = 0; b < kPollBatch; ++b)
                        if ((v[b] >> 32) != (tag >> 32)) v[b] = vb[base + 32 * b];
                }
#pragma unroll
                for (int b = 0; b < kPollBatch; ++b)
                    if (base + 32 * b < ti.size)
                        acc += __uint_as_float((unsigned)(v[b] & 0xffffffffull));
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
            ok = __all_sync(0xffffffffu, ok);
            if (lane == 0 && ok) {
                __threadfence();
                *reinterpret_cast<volatile unsigned long long*>(res) =
                    tag | (unsigned long long)__float_as_uint(acc);
            }
        }
        if (lane == 0) {
            unsigned long long v = 0;
            if (ok) {
                const volatile unsigned long long* vr = res;
                v = *vr;
                for (unsigned n = 1; (v >> 32) != (tag >> 32); ++n) {
                    if (timed_out(n)) { ok = false; break; }
                    __nanosleep(32);
                    v = *vr;
                }
            }
            __threadfence();
            s_tot = __uint_as_float((unsigned)(v & 0xffffffffull));
            s_ok = ok ? 1 : 0;
        }
    }
    __syncthreads();
    out = s_tot;
    const bool ok = s_ok != 0;
    __syncthreads();
    return ok;
}

// B items (slice tt, 8-site group) per thread and chunk: a chunk has
// nsl * 8 <= 512 items, so at most two per thread.
constexpr int kSkItems = 2;

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, uint32_t src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src),
                 "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Scale, split and store one B item (slice tt, group grp) into a chunk.
__device__ __forceinline__ void sk_store_item(const float4 (&v)[4], float scale, int Nn, int tt,
                                              int grp, uint8_t* chunk) {
    float re[8], im[8];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        re[2 * e] = v[e].x * scale;
        im[2 * e] = v[e].y * scale;
        re[2 * e + 1] = v[e].z * scale;
        im[2 * e + 1] = v[e].w * scale;
    }
    uint4 hr, lr, hm, lm;
    split8_plain(re, hr, lr);
    split8_plain(im, hm, lm);
    const int jr = 2 * tt, ji = jr + 1;
    uint8_t* lo = chunk + (size_t)Nn * 128;
    *reinterpret_cast<uint4*>(chunk + jr * 128 + ((grp ^ (jr & 7)) << 4)) = hr;
    *reinterpret_cast<uint4*>(lo + jr * 128 + ((grp ^ (jr & 7)) << 4)) = lr;
    *reinterpret_cast<uint4*>(chunk + ji * 128 + ((grp ^ (ji & 7)) << 4)) = hm;
    *reinterpret_cast<uint4*>(lo + ji * 128 + ((grp ^ (ji & 7)) << 4)) = lm;
}

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

// Build the stacked B of every chunk and issue the chunks' MMAs.  FP32
// source: every thread first issues cp.async copies of its 16-byte pieces
// of all chunks (raw layout [tt][64 sites] in the space of B chunk j; sites
// past V copy zeros, pieces past the K range are skipped), one commit group
// per chunk; then chunk by chunk it waits for the group, reads its items,
// and after a block barrier writes them split in place.  (Measured at
// L = 24: 5.5 us per application against 8.5 us with one bulk copy per
// slice row on the TMA engine.)  FP64 source (the residual after a reliable
// update): direct loads, chunk by chunk.
template <bool DAG>
__device__ __forceinline__ void sk_build_and_issue(const TcState& st, const SkGeom& g,
                                                   const SkSrc& src, int Nt, float scale,
                                                   uint32_t tmem) {
    const int Nn = g.Nn;
    uint8_t* bbase = st.base + g.b_off;
    const uint32_t chunk_bytes = 2u * (uint32_t)Nn * 128u;
    const int per_chunk = g.nsl * 8;
    const int kend = 16 * g.ks1;
    const int V = src.V;
    if (!src.use_d) {
        const int pieces = g.nsl * 32;   // 16-byte pieces (two sites) per chunk
#pragma unroll
        for (int j = 0; j < kSkMaxChunks; ++j) {
            if (j < g.nch) {
                const uint32_t raw = smem_u32(bbase + (size_t)j * chunk_bytes);
                for (int pc = threadIdx.x; pc < pieces; pc += blockDim.x) {
                    const int tt = pc >> 5, k = 16 * g.ks0 + KCH * j + 2 * (pc & 31);
                    if (k >= kend) continue;
                    const int ts = source_slice<DAG>(g.t0 + tt, Nt);
                    const bool in = k < V;     // V is even: a pair never straddles V
                    const float2* gp = src.f + (size_t)ts * V + (in ? k : 0);
                    cp_async16(raw + (uint32_t)pc * 16u, gp, in ? 16u : 0u);
                }
            }
            cp_async_commit();
        }
    }
#pragma unroll
    for (int j = 0; j < kSkMaxChunks; ++j) {
        if (j < g.nch) {
            uint8_t* ch = bbase + (size_t)j * chunk_bytes;
            float4 v[kSkItems][4];
            if (!src.use_d) {
                // the copies of chunks 0..j are complete for this thread
                if (j == 0) cp_async_wait<kSkMaxChunks - 1>();
                else if (j == 1) cp_async_wait<kSkMaxChunks - 2>();
                else if (j == 2) cp_async_wait<kSkMaxChunks - 3>();
                else cp_async_wait<0>();
                __syncthreads();
                const float4* raw = reinterpret_cast<const float4*>(ch);
#pragma unroll
                for (int m = 0; m < kSkItems; ++m) {
                    const int r = threadIdx.x + m * NTHR;
                    if (r < per_chunk) {
                        // item (tt, grp): 8 sites = 4 pieces of raw row tt
                        const int tt = r >> 3, grp = r & 7;
#pragma unroll
                        for (int e = 0; e < 4; ++e) v[m][e] = raw[tt * 32 + grp * 4 + e];
                    }
                }
                __syncthreads();   // every read of the raw chunk before the split overwrites it
            } else {
#pragma unroll
                for (int m = 0; m < kSkItems; ++m) {
                    const int r = threadIdx.x + m * NTHR;
                    const int kb = 16 * g.ks0 + KCH * j + 8 * (r & 7);
                    if (r < per_chunk && kb < kend) {
                        const int ts = source_slice<DAG>(g.t0 + (r >> 3), Nt);
                        const size_t o = (size_t)ts * V + kb;
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const float2 a =
                                kb + 2 * e < V ? src.one(o + 2 * e) : make_float2(0.f, 0.f);
                            const float2 b = kb + 2 * e + 1 < V ? src.one(o + 2 * e + 1)
                                                                : make_float2(0.f, 0.f);
                            v[m][e] = make_float4(a.x, a.y, b.x, b.y);
                        }
                    }
                }
            }
#pragma unroll
            for (int m = 0; m < kSkItems; ++m) {
                const int r = threadIdx.x + m * NTHR;
                const int kb = 16 * g.ks0 + KCH * j + 8 * (r & 7);
                if (r < per_chunk && kb < kend) sk_store_item(v[m], scale, Nn, r >> 3, r & 7, ch);
            }
            fence_proxy_async();
            __syncthreads();
            if (threadIdx.x == 0) sk_issue_chunk(st, g, j, smem_u32(ch), tmem);
        }
    }
}

// One split-K application: B from src (the source of every target slice of
// the n-group: t+1 for M^dag, t-1 for M) scaled by `scale`, the MMAs, the
// partial accumulator staged, a cluster sync, then this CTA's owned
// outputs: epi.store(tt, i, ow, w) gets w[4] = (E u)(i .. i+3) of slice
// t0 + tt (unscaled by 1/scale * 2^-eE), ow = the owner index of site i.
// All threads call it; false if a bounded wait failed (status set).
// The part of an application after the MMAs are issued: wait for the
// accumulator, stage it, sync the cluster (HW: the hardware cluster barrier
// of a standalone launch; else the bounded barrier of the CG team), sum the
// owned outputs' partials and run the epilogue.
template <bool HW, class Epi>
__device__ __forceinline__ bool sk_finish(TcState& st, const SkGeom& g, Team& tcl, int V,
                                          float unscale, Epi& epi) {
    TileBars& bars = *st.bars;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t tmem = bars.tmem_base;
    const int Nn = g.Nn;
    // partial accumulator -> staging [column][128 rows] (FP32)
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
            for (int e = 0; e < 16; ++e) stg[(cb * 16 + e) * TM + row] = m[e] + l[e];
        }
    }
    fence_before_sync();
    __syncthreads();
    if constexpr (HW) {
        cluster_barrier_all();   // every member's partial staged (release / acquire)
        if (!ok) return false;
    } else {
        if (!ok) return false;
        if (!sk_cluster_sync(tcl)) return false;
    }
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

template <bool DAG, class Epi>
__device__ __forceinline__ bool sk_apply(TcState& st, const SkGeom& g, Team& tcl,
                                         const SkSrc& src, int V, int Nt, float scale,
                                         float unscale, Epi& epi) {
    sk_build_and_issue<DAG>(st, g, src, Nt, scale, st.bars->tmem_base);
    return sk_finish<false>(st, g, tcl, V, unscale, epi);
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
// q = p' - s_{t+1} e^{-i phi_t} G,  u = e^{i phi_t} q.  Updates G, p (= p'),
// q in shared memory and writes u to global memory; sums |q|^2.
struct SkEpiDag {
    SkOwner ow;
    float2* u;
    const float2* cis;
    float beta;
    int V, Nt;
    float acc;
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
        const size_t o = (size_t)t * V + i;
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
            const float2 qv = make_float2(pv.x - sg * cg.x, pv.y - sg * cg.y);
            ow.G[oi + e] = gv;
            ow.p[oi + e] = pv;
            ow.q[oi + e] = qv;
            us[e] = cmulf(ph[e], qv);
            if (i + e < V) acc = fmaf(qv.x, qv.x, fmaf(qv.y, qv.y, acc));
        }
        if (i + 4 <= V) {
            *reinterpret_cast<float4*>(u + o) = make_float4(us[0].x, us[0].y, us[1].x, us[1].y);
            *reinterpret_cast<float4*>(u + o + 2) =
                make_float4(us[2].x, us[2].y, us[3].x, us[3].y);
        } else {
#pragma unroll
            for (int e = 0; e < 4; ++e)
                if (i + e < V) u[o + e] = us[e];
        }
    }
};

// M epilogue of the split-K CG iteration at (t, i .. i+3): with
// w = E u_{t-1},  Mq = q - s_t w,  x += alpha p,  r -= alpha Mq.  Updates x
// and r in shared memory, writes r to global memory; sums |r|^2.
struct SkEpiM {
    SkOwner ow;
    float2* r;
    float alpha;
    int V;
    float acc;
    __device__ __forceinline__ void prefetch(int, int) {}
    __device__ __forceinline__ void store(int t, int i, int oi, const float2 (&w)[4]) {
        const size_t o = (size_t)t * V + i;
        const float sg = (t == 0) ? -1.f : 1.f;
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
            if (i + e < V) acc = fmaf(rv.x, rv.x, fmaf(rv.y, rv.y, acc));
        }
        if (i + 4 <= V) {
            *reinterpret_cast<float4*>(r + o) = make_float4(rs[0].x, rs[0].y, rs[1].x, rs[1].y);
            *reinterpret_cast<float4*>(r + o + 2) =
                make_float4(rs[2].x, rs[2].y, rs[3].x, rs[3].y);
        } else {
#pragma unroll
            for (int e = 0; e < 4; ++e)
                if (i + e < V) r[o + e] = rs[e];
        }
    }
};

// Epilogue of a standalone application at (t, i .. i+3): with
// w = (E u)_t unscaled by the source slice's inverse scale inv[t] 2^-eE,
//     M:      out_t = in_t - s_t w                      (s_0 = -1)
//     M^dag:  out_t = in_t - s_{t+1} e^{-i phi_t} w     (s_Nt = -1)
template <bool DAG>
struct SkEpiOut {
    const float2* in;
    float2* out;
    const float2* cis;   // FP32 e^{i phi} (M^dag)
    const float* inv;    // per target slice
    float e_inv;
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
        const float u = inv[t] * e_inv;
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
            float2 wv = make_float2(w[e].x * u, w[e].y * u);
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
