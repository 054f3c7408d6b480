// tc_wide.cuh -- slice-major tensor-core tile of M or M^dag: the time slices
// are the MMA's M dimension and the sites its N dimension.
//
// GEMM view:  D[j][n] = sum_k U[j][k] E'[i0+n][k]
//   j = 2 tt + {0: re, 1: im}  for the tile's target slices t0 + tt, tt < 64
//                              (MMA M = 128),
//   n < W                      target sites of the tile (MMA N = W / nmma per
//                              instruction, nmma = 1 or 2),
//   k                          source site, K chunks of 64.
// U is the source of the tile's slices (e^{i phi_{t-1}} psi_{t-1} for M,
// psi_{t+1} for M^dag), the same rows the site-major tile builds.  A
// tcgen05.mma with M = 128 costs the same for every N up to 144 (measured:
// 78 cycles, the read of A), so putting the sites in N runs the tensor pipe
// at its full rate where the site-major tile (N = 2 x slices) pays that
// cost for 16 to 64 columns.
//
// Split precision with ONE FP32 accumulator:
//   E' = 2^eE E  = E'_hi + E'_lo   (fp16 each; lo is the plain remainder:
//                                   with max |E'| in [2^14, 2^15) it is
//                                   exact to 2^-24 absolute in fp16)
//   s u          = U_hi + U_lo     (s = 2^e puts |u| s in [2^12, 2^13); lo
//                                   again the plain remainder)
//   D = U_hi E'_hi + U_lo E'_hi + U_hi E'_lo = 2^eE s (E u) - U_lo E'_lo,
// the dropped term 2^-22 relative.  All three products accumulate into the
// same TMEM columns, so a tile holds up to 288 sites (TMEM: W columns).
//
// Ring stage s: [U_hi 16 KB][U_lo 16 KB][E'_hi W x 128 B][E'_lo W x 128 B],
// 128-byte-swizzled K-major rows.  Warp 0 loads E' (and, for a pre-split
// source, U) with TMA; warps 2..7 otherwise build U, one warp per slice with
// the lanes along the sites; warp 1 issues the MMAs.  The epilogue stages D
// through the (then idle) ring as [slice][site] rows and runs on all eight
// warps with the lanes along the sites, so its global traffic is contiguous
// over each warp (a thread per slice row would touch 16 cache lines per
// instruction).
#pragma once

#include "tc_tile.cuh"

namespace hmc {
namespace tc {

constexpr int WM = 128;                      // MMA M: 64 slices x {re, im}
constexpr int kWSlices = WM / 2;
constexpr int kWMaxW = 288;                  // sites per tile (TMEM columns)
constexpr int kWMaxN = 256;                  // MMA N per instruction
constexpr uint32_t kUTileBytes = WM * 128;   // one 64-wide K chunk of U_hi (or U_lo)
constexpr int kWMaxStages = 4;
constexpr int kMaxClusterW = 8;              // CTAs splitting one tile's K (portable cluster)
static_assert(kWMaxStages <= 4, "TileBars holds four slice-major stages");
static_assert(kWMaxW <= (int)kTmemCols, "one accumulator of W columns");
static_assert(2 * (2 * kUTileBytes + 2 * 128 * kWMaxW) <= kOperandBytes, "two wide stages");

// Geometry of the slice-major tiles of one operator: W sites per tile in
// nmma instructions of N = W / nmma, ring depth and stage size.
struct WideGeom {
    int W;
    int nmma;
    int stages;
    uint32_t stage_bytes;
};

__host__ __device__ inline WideGeom wide_geom(int W) {
    WideGeom g;
    g.W = W;
    g.nmma = W > kWMaxN ? 2 : 1;
    g.stage_bytes = 2 * kUTileBytes + 2 * 128u * (uint32_t)W;
    int s = (int)(kOperandBytes / g.stage_bytes);
    g.stages = s > kWMaxStages ? kWMaxStages : s;
    return g;
}

// Sites per slice-major tile for a lattice of V sites: every site in one
// tile up to 288 (N a multiple of 16 per instruction; two instructions of
// N = W/2 above 256), else tiles of 288.
__host__ __device__ inline int wide_sites(int V) {
    if (V > kWMaxW) return kWMaxW;
    int W = ((V + 15) / 16) * 16;
    if (W > kWMaxN) W = ((V + 31) / 32) * 32;   // two instructions of N = W/2
    return W;
}

// U chunk [k0, k0+64) of slices t0..t0+ns-1: one warp per slice, lane l
// holding sites k0 + 2l and k0 + 2l + 1 (one 16-byte load per source array,
// contiguous over the warp), split into fp16 hi and the plain remainder and
// written as four 32-bit words (re/im x hi/lo) into the swizzled rows 2 tt
// and 2 tt + 1.  Four slices per warp in flight (more made it slower: one
// SM's loads from L2 are bound by its bandwidth, not by their latency).  Rows of slices >= ns are
// left as they are (they only feed output rows the epilogue skips); sites
// >= V are zero (E' is zero there, U must be finite).  V is even, so a pair
// never straddles V.
template <bool DAG, class Src>
__device__ __forceinline__ void build_U(const Src& src, int V, int Nt, int t0, int ns, int k0,
                                        float scale, uint8_t* uhi, uint8_t* ulo, int pw,
                                        int lane) {
    const int k = k0 + 2 * lane;
    const uint32_t grp = (uint32_t)lane >> 2, wo = ((uint32_t)lane & 3u) * 4u;
    constexpr int UB = 4;
    for (int tb = pw; tb < ns; tb += UB * kNumBWarps) {
        float4 v[UB];
#pragma unroll
        for (int j = 0; j < UB; ++j) {
            const int tt = tb + j * kNumBWarps;
            v[j] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (tt < ns && k < V) v[j] = src.load2(source_slice<DAG>(t0 + tt, Nt), k);
        }
#pragma unroll
        for (int j = 0; j < UB; ++j) {
            const int tt = tb + j * kNumBWarps;
            if (tt < ns) {
                const float r0 = v[j].x * scale, i0 = v[j].y * scale;
                const float r1 = v[j].z * scale, i1 = v[j].w * scale;
                const __half rh0 = __float2half_rn(r0), rh1 = __float2half_rn(r1);
                const __half ih0 = __float2half_rn(i0), ih1 = __float2half_rn(i1);
                const __half rl0 = __float2half_rn(r0 - __half2float(rh0));
                const __half rl1 = __float2half_rn(r1 - __half2float(rh1));
                const __half il0 = __float2half_rn(i0 - __half2float(ih0));
                const __half il1 = __float2half_rn(i1 - __half2float(ih1));
                const uint32_t jr = 2u * (uint32_t)tt, ji = jr + 1u;
                const uint32_t orr = jr * 128u + ((grp ^ (jr & 7u)) << 4) + wo;
                const uint32_t oi = ji * 128u + ((grp ^ (ji & 7u)) << 4) + wo;
                *reinterpret_cast<uint32_t*>(uhi + orr) =
                    (uint32_t)__half_as_ushort(rh0) | ((uint32_t)__half_as_ushort(rh1) << 16);
                *reinterpret_cast<uint32_t*>(ulo + orr) =
                    (uint32_t)__half_as_ushort(rl0) | ((uint32_t)__half_as_ushort(rl1) << 16);
                *reinterpret_cast<uint32_t*>(uhi + oi) =
                    (uint32_t)__half_as_ushort(ih0) | ((uint32_t)__half_as_ushort(ih1) << 16);
                *reinterpret_cast<uint32_t*>(ulo + oi) =
                    (uint32_t)__half_as_ushort(il0) | ((uint32_t)__half_as_ushort(il1) << 16);
            }
        }
    }
}

// U prepared before the application (rows 2t / 2t+1 = re / im of the source
// of target slice t, fp16 hi and plain remainder, scaled by 1 / inv[t]); the
// TMA warp loads the tile's rows of it (a box of `rows` from row 2 t0; the
// MMA rows beyond keep stale data and feed only skipped outputs) with each
// E' chunk.
struct SrcSplitW {
    static constexpr bool kTma = true;
    const CUtensorMap* uhi;
    const CUtensorMap* ulo;
    const float* inv;
    int rows;     // TMA box rows of the U maps (2 x slices per tile, <= 128)
};

// Staged accumulator of a slice-major tile: FP32 complex rows [slice][site]
// at the start of the operand area, row stride W * 8 + 16 bytes (the two
// half-warps' rows fall on different banks).
__device__ __forceinline__ int wide_row_floats(int W) { return 2 * W + 4; }

// Contraction part of one slice-major tile: target slices t0..t0+ns-1
// (ns <= 64), sites i0..i0+W-1, K chunks [kc0, kc1).  Runs the ring (TMA,
// MMA, U producers), waits for the accumulator and stages it as FP32
// complex rows [slice][site] in the (then idle) ring.  Returns false if a
// bounded wait failed (status set).  All threads call it and leave it after
// a block barrier; the wide ring uses its own barriers and counters.
template <bool DAG, class Src>
__device__ bool tc_wstage(TcState& st, const WideGeom& g, const CUtensorMap* mhi,
                          const CUtensorMap* mlo, int V, int Nt, int i0, int t0, int ns,
                          int kc0, int kc1, const Src& src, float scale) {
    TileBars& bars = *st.bars;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nk = kc1 - kc0;
    const int W = g.W, Wm = W / g.nmma, S = g.stages;
    bool ok = true;
    // chunk j of the tile uses stage j % S (every tile starts at stage 0);
    // its fill index on that stage is wuse[s] + j / S
    uint32_t use0[kWMaxStages];
#pragma unroll
    for (int s = 0; s < kWMaxStages; ++s) use0[s] = st.wuse[s];
    auto stage = [&](uint32_t s) { return st.base + s * g.stage_bytes; };

    if (warp == kWarpTma) {
        if (lane == 0) {
            for (int j = 0; j < nk && ok; ++j) {
                const int kc = kc0 + j;
                const uint32_t s = (uint32_t)j % S, n = use0[s] + (uint32_t)j / S;
                if (n > 0) ok = mbar_wait(smem_u32(&bars.wempty[s]), (n - 1) & 1, st.status);
                if (!ok) break;
                const uint32_t bar = smem_u32(&bars.wfull[s]);
                const uint32_t u = smem_u32(stage(s));
                const uint32_t eh = u + 2 * kUTileBytes, el = eh + 128u * (uint32_t)W;
                uint32_t bytes = 256u * (uint32_t)W;
                if constexpr (Src::kTma) bytes += 2u * 128u * (uint32_t)src.rows;
                mbar_arrive_expect_tx(bar, bytes);
                for (int m = 0; m < g.nmma; ++m) {
                    const uint32_t o = (uint32_t)(m * Wm) * 128u;
                    tma_load_2d(eh + o, mhi, kc * KCH, i0 + m * Wm, bar);
                    tma_load_2d(el + o, mlo, kc * KCH, i0 + m * Wm, bar);
                }
                if constexpr (Src::kTma) {
                    tma_load_2d(u, src.uhi, kc * KCH, 2 * t0, bar);
                    tma_load_2d(u + kUTileBytes, src.ulo, kc * KCH, 2 * t0, bar);
                }
            }
        }
    } else if (warp == kWarpMma) {
        if (lane == 0) {
            const uint32_t idesc = idesc_f16(WM, Wm);
            const uint32_t tmem = bars.tmem_base;
            for (int j = 0; j < nk && ok; ++j) {
                const uint32_t s = (uint32_t)j % S, n = use0[s] + (uint32_t)j / S;
                ok = mbar_wait(smem_u32(&bars.wfull[s]), n & 1, st.status);
                if (!ok) break;
                fence_after_sync();
                const uint32_t uh = smem_u32(stage(s)), ul = uh + kUTileBytes;
                const uint32_t eh = uh + 2 * kUTileBytes, el = eh + 128u * (uint32_t)W;
#pragma unroll
                for (int kk = 0; kk < KCH / 16; ++kk) {
                    const uint32_t off = kk * 32;
                    const uint32_t acc = (j | kk) != 0;
                    for (int m = 0; m < g.nmma; ++m) {
                        const uint32_t bo = (uint32_t)(m * Wm) * 128u + off;
                        const uint32_t d = tmem + (uint32_t)(m * Wm);
                        mma_f16(d, desc_sw128(uh + off), desc_sw128(eh + bo), idesc, acc);
                        mma_f16(d, desc_sw128(ul + off), desc_sw128(eh + bo), idesc, 1u);
                        mma_f16(d, desc_sw128(uh + off), desc_sw128(el + bo), idesc, 1u);
                    }
                }
                mma_commit(smem_u32(&bars.wempty[s]));
            }
            mma_commit(smem_u32(&bars.wacc));
        }
    } else {
        // U producers (warps 2..7): each waits for the stage, builds its
        // items (unless the TMA loads U) and arrives once per chunk
        const int pw = warp - kFirstBWarp;
        for (int j = 0; j < nk && ok; ++j) {
            const int kc = kc0 + j;
            const uint32_t s = (uint32_t)j % S, n = use0[s] + (uint32_t)j / S;
            if (n > 0) ok = mbar_wait(smem_u32(&bars.wempty[s]), (n - 1) & 1, st.status);
            if (!ok) break;
            if constexpr (!Src::kTma) {
                uint8_t* uh = stage(s);
                build_U<DAG>(src, V, Nt, t0, ns, kc * KCH, scale, uh, uh + kUTileBytes, pw,
                             lane);
                fence_proxy_async();
            }
            __syncwarp();
            if (lane == 0)
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(
                                 smem_u32(&bars.wfull[s]))
                             : "memory");
        }
    }
    __syncwarp();
    // once the accumulator is complete the ring is free: stage D there
    if (ok) ok = mbar_wait(smem_u32(&bars.wacc), st.wtile & 1, st.status);
    fence_after_sync();
    ok = __all_sync(0xffffffffu, ok);   // tcgen05.ld below is warp-collective
    const int rs = wide_row_floats(W);
    float* ds = reinterpret_cast<float*>(st.base);
    if (ok) {
        // TMEM lane quarter q = warp % 4 (rows 32q..32q+31 = slices
        // 16q..16q+15); warps 4..7 the first half of the 16-site column
        // blocks, warps 0..3 the rest; lanes 2m, 2m+1 (re, im rows of one
        // slice) swap halves so each ends with 8 complete sites
        const int nb = W / 16, half = (nb + 1) / 2;
        const bool hi_warps = warp >= kFirstEpiWarp;
        const int b0 = hi_warps ? 0 : half, b1 = hi_warps ? half : nb;
        const int q = warp & 3, tt = (q * 32 + lane) >> 1;
        const bool odd = (lane & 1) != 0;
        const uint32_t tl = bars.tmem_base + ((uint32_t)(q * 32) << 16);
        for (int cb = b0; cb < b1; ++cb) {
            float v[16];
            tmem_ld16(tl + (uint32_t)(cb * 16), v);
            float o[16];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const float send = odd ? v[e] : v[8 + e];
                const float recv = __shfl_xor_sync(0xffffffffu, send, 1);
                o[2 * e] = odd ? recv : v[e];
                o[2 * e + 1] = odd ? v[8 + e] : recv;
            }
            float4* dst =
                reinterpret_cast<float4*>(ds + tt * rs + 2 * (cb * 16 + (odd ? 8 : 0)));
#pragma unroll
            for (int e = 0; e < 4; ++e)
                dst[e] = make_float4(o[4 * e], o[4 * e + 1], o[4 * e + 2], o[4 * e + 3]);
        }
    }
    for (int s = 0; s < S; ++s) st.wuse[s] += (uint32_t)((nk + S - 1 - s) / S);
    st.wtile += 1;
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    return ok;
}

// Epilogue of a slice-major tile from staged accumulators: segments of 64
// sites of one slice, dealt to the warps with the lanes along the sites, two
// sites per lane (Epi::load2 / store2: 16-byte accesses, so the epilogue's
// global traffic is contiguous over each warp in half the instructions),
// UN segments in flight per warp.  V and i0 are even, so a pair never
// straddles V.  With csize > 1 the tile's K was split over the csize CTAs of
// a thread-block cluster: this CTA (cluster rank `rank`) takes its share of
// the segments and sums the csize staged partials through distributed
// shared memory in rank order (deterministic); the caller brackets it with
// cluster barriers.
template <class Src, class Epi>
__device__ void tc_wepilogue(const TcState& st, int W, int V, int i0, int t0, int ns,
                             const Src& src, float inv_scale, float e_inv, Epi& epi, int rank,
                             int csize) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int rs = wide_row_floats(W);
    const float* ds = reinterpret_cast<const float*>(st.base);
    const uint32_t ds_s = smem_u32(ds);
    using In2 = typename Epi::In2;
    constexpr int UN = 2;
    const int nseg = (W + 63) / 64, total = ns * nseg;
    const int s0 = (int)((long long)total * rank / csize);
    const int s1 = (int)((long long)total * (rank + 1) / csize);
    for (int base = s0 + warp; base < s1; base += UN * (NTHR / 32)) {
        In2 in[UN];
#pragma unroll
        for (int u = 0; u < UN; ++u) {
            const int sg = base + u * (NTHR / 32);
            const int tt = sg / nseg, n = (sg - tt * nseg) * 64 + 2 * lane;
            if (sg < s1 && n < W && i0 + n < V) in[u] = epi.load2(i0 + n, t0 + tt);
        }
#pragma unroll
        for (int u = 0; u < UN; ++u) {
            const int sg = base + u * (NTHR / 32);
            const int tt = sg / nseg, n = (sg - tt * nseg) * 64 + 2 * lane;
            if (sg < s1 && n < W && i0 + n < V) {
                float is = inv_scale * e_inv;
                if constexpr (Src::kTma) is = src.inv[t0 + tt] * e_inv;
                float4 d;
                if (csize == 1) {
                    d = *reinterpret_cast<const float4*>(ds + tt * rs + 2 * n);
                } else {
                    d = make_float4(0.f, 0.f, 0.f, 0.f);
                    const uint32_t off = ds_s + (uint32_t)((tt * rs + 2 * n) * 4);
                    // non-volatile loads (the sums may trail them, so the
                    // members' loads can be in flight together); the memory
                    // clobber keeps them after the caller's cluster barrier
                    float4 x[kMaxClusterW];
#pragma unroll
                    for (int qr = 0; qr < kMaxClusterW; ++qr) {
                        if (qr < csize) {
                            uint32_t ra;
                            asm("mapa.shared::cluster.u32 %0, %1, %2;"
                                : "=r"(ra)
                                : "r"(off), "r"(qr));
                            asm("ld.shared::cluster.v4.f32 {%0, %1, %2, %3}, [%4];"
                                : "=f"(x[qr].x), "=f"(x[qr].y), "=f"(x[qr].z), "=f"(x[qr].w)
                                : "r"(ra)
                                : "memory");
                        }
                    }
#pragma unroll
                    for (int qr = 0; qr < kMaxClusterW; ++qr) {
                        if (qr < csize) {
                            d.x += x[qr].x;
                            d.y += x[qr].y;
                            d.z += x[qr].z;
                            d.w += x[qr].w;
                        }
                    }
                }
                epi.store2(i0 + n, t0 + tt, in[u], make_float2(d.x * is, d.y * is),
                           make_float2(d.z * is, d.w * is));
            }
        }
    }
}

// One slice-major tile on one CTA: contraction over all K, then the
// epilogue.  Epi::load / Epi::store as for tc_tile; store receives
// w = (E u)_i for the source of target slice t.  e_inv = 2^-eE undoes the
// scale of E'.  Returns false if a bounded wait failed (status set).  All
// threads call it.
template <bool DAG, class Src, class Epi>
__device__ bool tc_wtile(TcState& st, const WideGeom& g, const CUtensorMap* mhi,
                         const CUtensorMap* mlo, int V, int Nt, int Vp, int i0, int t0, int ns,
                         const Src& src, float scale, float inv_scale, float e_inv, Epi& epi) {
    tc_wstage<DAG>(st, g, mhi, mlo, V, Nt, i0, t0, ns, 0, Vp / KCH, src, scale);
    if (*((volatile int*)st.status) == 0)
        tc_wepilogue(st, g.W, V, i0, t0, ns, src, inv_scale, e_inv, epi, 0, 1);
    fence_proxy_async();   // the next tile's TMA writes where D was staged
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    return *((volatile int*)st.status) == 0;
}

}  // namespace tc
}  // namespace hmc
