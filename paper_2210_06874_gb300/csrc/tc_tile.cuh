// tc_tile.cuh -- one output tile of M or M^dag on the sm_103a tensor cores.
//
// GEMM view of the hopping contraction: D[i][j] = sum_k E[i][k] B[j][k],
// i = site (MMA M = 128 per tile), j = 2*slice + {re, im} (MMA N = 2 * slices
// of the tile), k = source site.  Split precision (FP16 operands, FP32
// accumulation):
//     E      = E_hi + 2^-11 E_lo          (host-made split, streamed by TMA)
//     v s    = B_hi + 2^-11 B_lo          (built here; s = 2^e scales the vector
//                                          so that |v| s is in [2^12, 2^13))
//     E v s ~= E_hi B_hi + 2^-11 (E_hi B_lo + E_lo B_hi)
// accumulated in two TMEM accumulators (main at column 0, correction at
// column 128).  The dropped E_lo B_lo term is 2^-22 relative.
//
// B is built by the CTA's threads straight into the 128-byte-swizzled
// K-major layout the MMA reads: for M the phase exp(i phi_{t-1}) is
// multiplied in; for M^dag the source slice is t+1 and the conjugate phase
// of the target slice is applied in the epilogue.  Two pipeline stages: while
// the MMAs of chunk k run, the TMA of E and the B build of chunk k+1 fill the
// other stage.
#pragma once

#include "tc_ptx.cuh"

namespace hmc {
namespace tc {

constexpr int TM = 128;         // sites per tile (MMA M)
constexpr int KCH = 64;         // K per chunk: one 128-byte swizzle row of fp16
constexpr int NMAX = 128;       // max MMA N (= 2 * slices per tile)
constexpr int NTHR = 256;       // threads per CTA
constexpr int kStages = 2;
constexpr uint32_t kTmemCols = 256;    // main accumulator at 0, correction at 128
constexpr uint32_t kCorrCol = 128;
constexpr float kLoScale = 2048.f;     // 2^11
constexpr float kLoInv = 1.f / 2048.f;
constexpr uint32_t kATileBytes = TM * 128;

struct TileSmem {
    uint8_t a_hi[kStages][TM * 128];
    uint8_t a_lo[kStages][TM * 128];
    uint8_t b_hi[kStages][NMAX * 128];
    uint8_t b_lo[kStages][NMAX * 128];
    uint64_t tma_bar[kStages];
    uint64_t mma_bar[kStages];
    uint32_t tmem_base;
    int ok;
};
constexpr size_t kSmemBytes = sizeof(TileSmem) + 1024;  // + alignment slack

__device__ __forceinline__ TileSmem& tile_smem(uint8_t* dyn) {
    const uint32_t a = smem_u32(dyn);
    return *reinterpret_cast<TileSmem*>(dyn + ((1024u - (a & 1023u)) & 1023u));
}

// Split 8 floats into fp16 hi and fp16 (x - hi) * 2^11, packed 8 per uint4.
__device__ __forceinline__ void split8(const float (&x)[8], uint4& hi, uint4& lo) {
    uint32_t h[4], l[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const __half h0 = __float2half_rn(x[2 * e]);
        const __half h1 = __float2half_rn(x[2 * e + 1]);
        const __half l0 = __float2half_rn((x[2 * e] - __half2float(h0)) * kLoScale);
        const __half l1 = __float2half_rn((x[2 * e + 1] - __half2float(h1)) * kLoScale);
        h[e] = (uint32_t)__half_as_ushort(h0) | ((uint32_t)__half_as_ushort(h1) << 16);
        l[e] = (uint32_t)__half_as_ushort(l0) | ((uint32_t)__half_as_ushort(l1) << 16);
    }
    hi = make_uint4(h[0], h[1], h[2], h[3]);
    lo = make_uint4(l[0], l[1], l[2], l[3]);
}

// Source slice of target slice t: t-1 for M, t+1 for M^dag (mod Nt).
template <bool DAG>
__device__ __forceinline__ int source_slice(int t, int Nt) {
    return DAG ? (t + 1 == Nt ? 0 : t + 1) : (t == 0 ? Nt - 1 : t - 1);
}

// Fill the B operand of K chunk [k0, k0+64) for the tile's slices t0..t0+ns-1
// (rows 2*tt (re) and 2*tt+1 (im); rows up to nrows-1 beyond 2*ns are zero).
template <bool DAG>
__device__ __forceinline__ void build_B(const float2* __restrict__ in,
                                        const float2* __restrict__ cis, int V, int Nt, int t0,
                                        int ns, int nrows, int k0, float scale, uint8_t* bhi,
                                        uint8_t* blo) {
    const int items = (nrows >> 1) * 8;
    for (int w = threadIdx.x; w < items; w += NTHR) {
        const int tt = w >> 3, grp = w & 7;
        const int kb = k0 + grp * 8;
        float re[8], im[8];
        if (tt < ns) {
            const int ts = source_slice<DAG>(t0 + tt, Nt);
            const float2* src = in + (size_t)ts * V + kb;
            const float2* ph = cis + (size_t)ts * V + kb;
            float2 v[8];
            if (kb + 8 <= V) {
                const float4* s4 = reinterpret_cast<const float4*>(src);
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const float4 a = s4[e];
                    v[2 * e] = make_float2(a.x, a.y);
                    v[2 * e + 1] = make_float2(a.z, a.w);
                }
                if (!DAG) {
                    const float4* p4 = reinterpret_cast<const float4*>(ph);
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const float4 a = p4[e];
                        v[2 * e] = cmulf(make_float2(a.x, a.y), v[2 * e]);
                        v[2 * e + 1] = cmulf(make_float2(a.z, a.w), v[2 * e + 1]);
                    }
                }
            } else {
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    v[e] = make_float2(0.f, 0.f);
                    if (kb + e < V) {
                        v[e] = src[e];
                        if (!DAG) v[e] = cmulf(ph[e], v[e]);
                    }
                }
            }
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                re[e] = v[e].x * scale;
                im[e] = v[e].y * scale;
            }
        } else {
#pragma unroll
            for (int e = 0; e < 8; ++e) re[e] = im[e] = 0.f;
        }
        uint4 hr, lr, hm, lm;
        split8(re, hr, lr);
        split8(im, hm, lm);
        const int jr = 2 * tt, ji = jr + 1;
        *reinterpret_cast<uint4*>(bhi + jr * 128 + ((grp ^ (jr & 7)) << 4)) = hr;
        *reinterpret_cast<uint4*>(blo + jr * 128 + ((grp ^ (jr & 7)) << 4)) = lr;
        *reinterpret_cast<uint4*>(bhi + ji * 128 + ((grp ^ (ji & 7)) << 4)) = hm;
        *reinterpret_cast<uint4*>(blo + ji * 128 + ((grp ^ (ji & 7)) << 4)) = lm;
    }
}

// Per-CTA state of the tensor-core tile pipeline (set up once per launch).
struct TcState {
    TileSmem* sm;
    uint32_t gchunk;   // chunks processed so far by this CTA (mbarrier phases)
    int* status;
};

// One-time set-up: mbarriers and TMEM.  All threads call it.
__device__ inline void tc_setup(TcState& st, uint8_t* dyn, int* status) {
    TileSmem& sm = tile_smem(dyn);
    st.sm = &sm;
    st.gchunk = 0;
    st.status = status;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(smem_u32(&sm.tma_bar[s]), 1);
            mbar_init(smem_u32(&sm.mma_bar[s]), 1);
        }
        fence_mbar_init();
    }
    if ((threadIdx.x >> 5) == 0) {
        tmem_alloc(smem_u32(&sm.tmem_base), kTmemCols);
        tmem_relinquish();
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
}

// Tear-down: wait (bounded) for the last MMAs, free TMEM.  All threads call it.
__device__ inline void tc_teardown(TcState& st) {
    TileSmem& sm = *st.sm;
    if (st.gchunk > 0) {
        const uint32_t g = st.gchunk - 1;
        mbar_wait(smem_u32(&sm.mma_bar[g & 1]), (g >> 1) & 1, st.status);
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    if ((threadIdx.x >> 5) == 0) tmem_dealloc(sm.tmem_base, kTmemCols);
}

// Scale 2^e with |v| 2^e in [2^12, 2^13) for a vector of squared norm n2.
__device__ __forceinline__ void vector_scale(double n2, float& scale, float& inv) {
    int e = 0;
    if (n2 > 0.0 && isfinite(n2)) {
        e = 12 - ilogb(sqrt(n2));
        e = max(-120, min(120, e));
    }
    scale = ldexpf(1.f, e);
    inv = ldexpf(1.f, -e);
}

// One output tile: target slices t0 .. t0+ns-1 (ns <= NMAX/2), sites
// i0 .. i0+127.  Epi(i, t, w) receives w = (E u)_{i} for the tile's source
// slice of target t (unscaled, before shift sign and phase).  Returns false
// if a bounded wait failed (status set).  All threads call it.
template <bool DAG, class Epi>
__device__ bool tc_tile(TcState& st, const CUtensorMap* mhi, const CUtensorMap* mlo, int V,
                        int Nt, int Vp, int i0, int t0, int ns, const float2* in,
                        const float2* cis, float scale, float inv_scale, Epi& epi) {
    TileSmem& sm = *st.sm;
    const int tid = threadIdx.x;
    const int nk = Vp / KCH;
    const int N = ((2 * ns + 15) / 16) * 16;
    const uint32_t idesc = idesc_f16(TM, N);
    const uint32_t tmem = sm.tmem_base;
    bool ok = true;
    const uint32_t g0 = st.gchunk;

    auto fill = [&](int kc, uint32_t g) {
        const int s = g & 1;
        if (g >= 2 && ok) ok = mbar_wait(smem_u32(&sm.mma_bar[s]), ((g - 2) >> 1) & 1, st.status);
        if (tid == 0 && ok) {
            const uint32_t bar = smem_u32(&sm.tma_bar[s]);
            mbar_arrive_expect_tx(bar, 2 * kATileBytes);
            tma_load_2d(smem_u32(sm.a_hi[s]), mhi, kc * KCH, i0, bar);
            tma_load_2d(smem_u32(sm.a_lo[s]), mlo, kc * KCH, i0, bar);
        }
        if (ok)
            build_B<DAG>(in, cis, V, Nt, t0, ns, N, kc * KCH, scale, sm.b_hi[s], sm.b_lo[s]);
        fence_proxy_async();
    };

    fill(0, g0);
    __syncthreads();
    for (int kc = 0; kc < nk; ++kc) {
        const uint32_t g = g0 + kc;
        const int s = g & 1;
        if (tid == 0 && ok) {
            ok = mbar_wait(smem_u32(&sm.tma_bar[s]), (g >> 1) & 1, st.status);
            if (ok) {
                fence_after_sync();
                const uint32_t ah = smem_u32(sm.a_hi[s]), al = smem_u32(sm.a_lo[s]);
                const uint32_t bh = smem_u32(sm.b_hi[s]), bl = smem_u32(sm.b_lo[s]);
#pragma unroll
                for (int kk = 0; kk < KCH / 16; ++kk) {
                    const uint32_t off = kk * 32;
                    const uint32_t acc = (kc | kk) != 0;
                    mma_f16(tmem, desc_sw128(ah + off), desc_sw128(bh + off), idesc, acc);
                    mma_f16(tmem + kCorrCol, desc_sw128(ah + off), desc_sw128(bl + off), idesc,
                            acc);
                    mma_f16(tmem + kCorrCol, desc_sw128(al + off), desc_sw128(bh + off), idesc,
                            1u);
                }
                mma_commit(smem_u32(&sm.mma_bar[s]));
            }
        }
        if (kc + 1 < nk) fill(kc + 1, g + 1);
        __syncthreads();
    }
    st.gchunk = g0 + nk;
    {
        const uint32_t g = g0 + nk - 1;
        if (ok) ok = mbar_wait(smem_u32(&sm.mma_bar[g & 1]), (g >> 1) & 1, st.status);
    }
    fence_after_sync();
    // epilogue: warp w reads TMEM lanes 32*(w%4).., column blocks of 16
    const int warp = tid >> 5, lane = tid & 31;
    const int row = (warp & 3) * 32 + lane;
    const int i = i0 + row;
    const uint32_t tl = tmem + ((uint32_t)((warp & 3) * 32) << 16);
    if (ok) {
        for (int cb = (warp >> 2) * 16; cb < N; cb += 32) {
            float m[16], c[16];
            tmem_ld16(tl + cb, m);
            tmem_ld16(tl + kCorrCol + cb, c);
            if (i < V) {
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const int tt = (cb >> 1) + e;
                    if (tt < ns) {
                        const float wr = fmaf(c[2 * e], kLoInv, m[2 * e]) * inv_scale;
                        const float wi = fmaf(c[2 * e + 1], kLoInv, m[2 * e + 1]) * inv_scale;
                        epi(i, t0 + tt, make_float2(wr, wi));
                    }
                }
            }
        }
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    return ok && (*((volatile int*)st.status) == 0);
}

}  // namespace tc
}  // namespace hmc
