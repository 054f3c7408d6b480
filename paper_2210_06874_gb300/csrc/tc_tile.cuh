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
// column 64).  The dropped E_lo B_lo term is 2^-22 relative.
//
// B is built by six warps straight into the 128-byte-swizzled K-major
// layout the MMA reads: for M the phase exp(i phi_{t-1}) is multiplied in;
// for M^dag the source slice is t+1 and the conjugate phase of the target
// slice is applied in the epilogue.  A ring of operand stages with full/empty
// mbarriers keeps TMA, B production and MMA issue overlapped.  In resident
// mode the CTA's rows of E_hi/E_lo (all K) stay in shared memory for a whole
// solve and only B streams through the ring.
#pragma once

#include "tc_ptx.cuh"

namespace hmc {
namespace tc {

constexpr int TM = 128;         // sites per tile (MMA M)
constexpr int KCH = 64;         // K per chunk: one 128-byte swizzle row of fp16
constexpr int NMAX = 64;        // max MMA N (= 2 * slices per tile)
constexpr int NTHR = 256;       // threads per CTA (8 warps)
constexpr int kMaxStages = 4;   // deepest operand ring
constexpr uint32_t kTmemCols = 512;    // site-major tile: main at 0, correction at 64;
                                       // slice-major tile (tc_wide.cuh): W columns
constexpr uint32_t kCorrCol = 64;
constexpr float kLoScale = 2048.f;     // 2^11
constexpr float kLoInv = 1.f / 2048.f;
constexpr uint32_t kATileBytes = TM * 128;          // one 64-wide K chunk of E_hi (or E_lo)
constexpr uint32_t kAChunkBytes = 2 * kATileBytes;  // E_hi + E_lo
constexpr uint32_t kBTileBytes = NMAX * 128;        // one chunk of B_hi (or B_lo)
constexpr uint32_t kBStageBytes = 2 * kBTileBytes;  // streaming B stage (N <= 64)
constexpr uint32_t kBStageSmall = kBStageBytes / 2; // resident B stage (N <= 32)
constexpr uint32_t kOperandBytes = 208 * 1024;      // operand area of dynamic smem
constexpr int kMaxResidentChunks = 4;               // resident E: K <= 256
// warp roles
constexpr int kWarpTma = 0;            // lane 0 issues the TMA loads of E
constexpr int kWarpMma = 1;            // lane 0 issues tcgen05.mma
constexpr int kFirstBWarp = 2;         // warps 2..7 build the B operand
constexpr int kNumBWarps = 6;
constexpr int kFirstEpiWarp = 4;       // warps 4..7 read TMEM (lane quarter = warp % 4)
static_assert((NMAX / 2) * 8 <= 2 * kNumBWarps * 32, "build_B covers at most 2 items/thread");
static_assert(kNumBWarps % 6 == 0, "producer groups of 1, 2 or 3");
static_assert(kMaxStages * (kAChunkBytes + kBStageBytes) <= kOperandBytes, "streaming ring");
static_assert(kMaxResidentChunks * kAChunkBytes + kMaxStages * kBStageSmall <= kOperandBytes,
              "resident E + B ring");

// Barriers and the TMEM address follow the operand area.
struct TileBars {
    uint64_t full[kMaxStages];    // B producers (+ TMA bytes when streaming)
    uint64_t empty[kMaxStages];   // MMA commit: the stage may be refilled
    uint64_t acc_full;            // MMA commit after a tile's last chunk
    uint64_t res_full;            // resident E landed
    uint64_t wfull[4];            // slice-major ring (tc_wide.cuh): TMA bytes + producers
    uint64_t wempty[4];           // slice-major ring: MMA commit
    uint64_t wacc;                // slice-major tile: accumulator complete
    uint64_t skb[4];              // split-K standalone application: B chunk j landed
    uint32_t tmem_base;
};
constexpr size_t kSmemBytes = kOperandBytes + sizeof(TileBars) + 1024;  // + alignment slack

// Operand layouts of the dynamic shared memory (1024-byte aligned base);
// four ring stages in the two tensor-core layouts:
//   streaming: stage s holds E_hi/E_lo chunk (32 KB) at s*32K and the B
//              stage (16 KB, N <= 64) at 128K + s*16K; E streamed by TMA
//   resident:  E_hi/E_lo of all nk K chunks of the CTA's site block at
//              kc*32K (loaded once per solve), B stages (8 KB, N <= 32) at
//              nk*32K + s*8K; the rest of the area can hold the FP32 CG
//              vectors of a chain that one CTA solves alone
//   small:     no tensor-core tiles; the CUDA-core cluster solver of
//              small_cg.cuh lays out E^T and its vectors in the area
//   slice:     slice-major tiles (tc_wide.cuh): a ring of U + E' stages
//              from the start of the area, with its own barriers
//   splitk:    split-K tiles (tc_splitk.cuh): the CTA's rows x K range of
//              E' resident (loaded once per launch), the stacked B of its
//              chunks, and the staged partial accumulator
enum OperandMode : int { kStreaming = 0, kResident = 1, kSmall = 2, kSlice = 3, kSplitK = 4 };

__device__ __forceinline__ uint8_t* smem_base(uint8_t* dyn) {
    const uint32_t a = smem_u32(dyn);
    return dyn + ((1024u - (a & 1023u)) & 1023u);
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

// Sources of the B operand: value of the vector the tile contracts with E,
// at source slice ts and sites kb..kb+7 (kb a multiple of 8, kb + 8 <= V)
// or at one site k.
struct SrcPlain {                       // u = in
    static constexpr bool kTma = false;
    const float2* in;
    int V;
    __device__ __forceinline__ void load8(int ts, int kb, float2 (&v)[8]) const {
        const float4* s4 = reinterpret_cast<const float4*>(in + (size_t)ts * V + kb);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const float4 a = s4[e];
            v[2 * e] = make_float2(a.x, a.y);
            v[2 * e + 1] = make_float2(a.z, a.w);
        }
    }
    __device__ __forceinline__ float2 load1(int ts, int k) const { return in[(size_t)ts * V + k]; }
    // sites k, k+1 (k even, k + 1 < V): one 16-byte load
    __device__ __forceinline__ float4 load2(int ts, int k) const {
        return *reinterpret_cast<const float4*>(in + (size_t)ts * V + k);
    }
};

struct SrcPhase {                       // u = exp(i phi) * in
    static constexpr bool kTma = false;
    const float2* in;
    const float2* cis;
    int V;
    __device__ __forceinline__ void load8(int ts, int kb, float2 (&v)[8]) const {
        const float4* s4 = reinterpret_cast<const float4*>(in + (size_t)ts * V + kb);
        const float4* p4 = reinterpret_cast<const float4*>(cis + (size_t)ts * V + kb);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const float4 a = s4[e], c = p4[e];
            v[2 * e] = cmulf(make_float2(c.x, c.y), make_float2(a.x, a.y));
            v[2 * e + 1] = cmulf(make_float2(c.z, c.w), make_float2(a.z, a.w));
        }
    }
    __device__ __forceinline__ float2 load1(int ts, int k) const {
        const size_t o = (size_t)ts * V + k;
        return cmulf(cis[o], in[o]);
    }
    __device__ __forceinline__ float4 load2(int ts, int k) const {
        const size_t o = (size_t)ts * V + k;
        const float4 a = *reinterpret_cast<const float4*>(in + o);
        const float4 c = *reinterpret_cast<const float4*>(cis + o);
        const float2 u0 = cmulf(make_float2(c.x, c.y), make_float2(a.x, a.y));
        const float2 u1 = cmulf(make_float2(c.z, c.w), make_float2(a.z, a.w));
        return make_float4(u0.x, u0.y, u1.x, u1.y);
    }
};

// u = p_new = r + beta p_old, the CG direction update done on the fly; r is
// the FP32 iterate, or (refresh) the FP64 true residual rounded to FP32.
struct SrcDirection {
    static constexpr bool kTma = false;
    const float2* r;
    const double2* r64;
    const float2* p_old;
    float beta;
    bool refresh;
    int V;
    __device__ __forceinline__ float2 one(size_t o) const {
        float2 rv;
        if (refresh) {
            const double2 d = r64[o];
            rv = make_float2((float)d.x, (float)d.y);
        } else {
            rv = r[o];
        }
        const float2 pv = p_old[o];
        return make_float2(fmaf(beta, pv.x, rv.x), fmaf(beta, pv.y, rv.y));
    }
    __device__ __forceinline__ void load8(int ts, int kb, float2 (&v)[8]) const {
        const size_t o = (size_t)ts * V + kb;
        if (refresh) {
#pragma unroll
            for (int e = 0; e < 8; ++e) v[e] = one(o + e);
            return;
        }
        const float4* r4 = reinterpret_cast<const float4*>(r + o);
        const float4* p4 = reinterpret_cast<const float4*>(p_old + o);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const float4 a = r4[e], b = p4[e];
            v[2 * e] = make_float2(fmaf(beta, b.x, a.x), fmaf(beta, b.y, a.y));
            v[2 * e + 1] = make_float2(fmaf(beta, b.z, a.z), fmaf(beta, b.w, a.w));
        }
    }
    __device__ __forceinline__ float2 load1(int ts, int k) const {
        return one((size_t)ts * V + k);
    }
    __device__ __forceinline__ float4 load2(int ts, int k) const {
        const size_t o = (size_t)ts * V + k;
        if (refresh) {
            const float2 a = one(o), b = one(o + 1);
            return make_float4(a.x, a.y, b.x, b.y);
        }
        const float4 a = *reinterpret_cast<const float4*>(r + o);
        const float4 b = *reinterpret_cast<const float4*>(p_old + o);
        return make_float4(fmaf(beta, b.x, a.x), fmaf(beta, b.y, a.y), fmaf(beta, b.z, a.z),
                           fmaf(beta, b.w, a.w));
    }
};

// B prepared before the application (one FP16 hi/lo split per time slice,
// rows 2t / 2t+1 = re / im of the source of target slice t, K contiguous,
// scaled by the power of two 1 / inv[t]): the TMA warp loads it with the
// E chunk, the producer warps only keep the barrier count, and the
// epilogue unscales column by column.
struct SrcSplit {
    static constexpr bool kTma = true;
    const CUtensorMap* bhi;
    const CUtensorMap* blo;
    const float* inv;
    int rows;     // TMA box rows of B (the MMA N of every tile, the last ragged one too)
};

// Fill the B operand of K chunk [k0, k0+64) for the tile's slices t0..t0+ns-1
// (rows 2*tt (re) and 2*tt+1 (im); rows up to nrows-1 beyond 2*ns are zero).
template <bool DAG, class Src>
__device__ __forceinline__ void build_B(const Src& src, int V, int Nt, int t0, int ns,
                                        int nrows, int k0, float scale, uint8_t* bhi,
                                        uint8_t* blo, int ptid, int nprod) {
    const int items = (nrows >> 1) * 8;
    // at most two items per producer thread (nrows <= 64, 192 producers):
    // issue the global loads of both before converting either
    float2 v[2][8];
    int wi[2];
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        const int w = ptid + j * nprod;
        wi[j] = w;
        if (w >= items) continue;
        const int tt = w >> 3, kb = k0 + (w & 7) * 8;
        if (tt < ns) {
            const int ts = source_slice<DAG>(t0 + tt, Nt);
            if (kb + 8 <= V) {
                src.load8(ts, kb, v[j]);
            } else {
#pragma unroll
                for (int e = 0; e < 8; ++e)
                    v[j][e] = (kb + e < V) ? src.load1(ts, kb + e) : make_float2(0.f, 0.f);
            }
        } else {
#pragma unroll
            for (int e = 0; e < 8; ++e) v[j][e] = make_float2(0.f, 0.f);
        }
    }
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        const int w = wi[j];
        if (w >= items) continue;
        const int tt = w >> 3, grp = w & 7;
        float re[8], im[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            re[e] = v[j][e].x * scale;
            im[e] = v[j][e].y * scale;
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

// Resident B (tile argument res_b != 0, streaming layout): the B operand of
// all K chunks of a slice tile, hi chunks then lo chunks of N x 128 bytes,
// in the area after the E ring.
__host__ __device__ constexpr size_t res_b_bytes(int N, int Vp) {
    return 2 * (size_t)(Vp / KCH) * (size_t)N * 128;
}
constexpr size_t kResBArea = kOperandBytes - (size_t)kMaxStages * kAChunkBytes;

// Per-CTA state of the tensor-core tile pipeline (set up once per launch).
struct TcState {
    uint8_t* base;     // 1024-aligned operand area
    TileBars* bars;
    int mode;          // OperandMode
    int stages;        // ring depth
    uint32_t b_off;    // offset of the B ring
    uint32_t b_stage;  // bytes per B stage (B_hi then B_lo, half each)
    uint32_t gchunk;   // chunks processed so far by this CTA (ring phases)
    uint32_t ntile;    // tiles processed so far (accumulator phases)
    uint32_t nres;     // resident loads so far (phases of res_full)
    uint32_t wuse[4];  // slice-major ring: fills of each stage so far (the ring
                       // depth depends on the tile width, so each stage's
                       // barrier phases are counted on their own)
    uint32_t wtile;    // slice-major tiles so far
    uint32_t gseq;     // split-K: team words posted so far (sk_post)
    int sk_loaded;     // split-K: this CTA's part of E' is resident
    uint32_t nskb;     // split-K CG: applications whose sources came by TMA (skb phases)
    int* status;
    __device__ __forceinline__ uint8_t* a_hi(int kc, int s) const {
        return base + (mode == kResident ? kc : s) * kAChunkBytes;
    }
    __device__ __forceinline__ uint8_t* b_hi(int s) const {
        return base + b_off + s * b_stage;
    }
    // first byte after the B ring (free for resident vectors)
    __device__ __forceinline__ uint8_t* free_area() const {
        return base + b_off + stages * b_stage;
    }
};

// One-time set-up: mbarriers and TMEM, streaming layout.  All threads.
__device__ inline void tc_setup(TcState& st, uint8_t* dyn, int* status) {
    st.base = smem_base(dyn);
    st.bars = reinterpret_cast<TileBars*>(st.base + kOperandBytes);
    st.mode = kStreaming;
    st.stages = kMaxStages;
    st.b_off = kMaxStages * kAChunkBytes;
    st.b_stage = kBStageBytes;
    st.gchunk = 0;
    st.ntile = 0;
    st.nres = 0;
    for (int s = 0; s < 4; ++s) st.wuse[s] = 0;
    st.wtile = 0;
    st.gseq = 0;
    st.sk_loaded = 0;
    st.nskb = 0;
    st.status = status;
    TileBars& b = *st.bars;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kMaxStages; ++s) {
            mbar_init(smem_u32(&b.full[s]), 1 + kNumBWarps);
            mbar_init(smem_u32(&b.empty[s]), 1);
        }
        mbar_init(smem_u32(&b.acc_full), 1);
        mbar_init(smem_u32(&b.res_full), 1);
        for (int j = 0; j < 4; ++j) mbar_init(smem_u32(&b.skb[j]), 1);
        for (int s = 0; s < 4; ++s) {
            mbar_init(smem_u32(&b.wfull[s]), 1 + kNumBWarps);
            mbar_init(smem_u32(&b.wempty[s]), 1);
        }
        mbar_init(smem_u32(&b.wacc), 1);
        fence_mbar_init();
    }
    if ((threadIdx.x >> 5) == 0) {
        tmem_alloc(smem_u32(&b.tmem_base), kTmemCols);
        tmem_relinquish();
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
}

// Choose the operand layout.  The ring depth is the same in both modes, so
// the layout may change between solves or chains (no chunk is in flight
// then: every tile waits for its accumulator before returning).
__device__ inline void tc_set_layout(TcState& st, int mode, int nk) {
    st.mode = mode;
    if (mode == kResident) {
        st.b_off = nk * kAChunkBytes;
        st.b_stage = kBStageSmall;
    } else {
        st.b_off = kMaxStages * kAChunkBytes;
        st.b_stage = kBStageBytes;
    }
}

// Resident mode: load E_hi/E_lo rows i0..i0+127, all nk K chunks, into the
// operand area with TMA and wait (bounded).  All threads call it, between
// tiles.
__device__ inline bool tc_load_resident(TcState& st, const CUtensorMap* mhi,
                                        const CUtensorMap* mlo, int i0, int nk) {
    TileBars& b = *st.bars;
    tc_set_layout(st, kResident, nk);
    __syncthreads();
    if (threadIdx.x == 0) {
        const uint32_t bar = smem_u32(&b.res_full);
        mbar_arrive_expect_tx(bar, nk * kAChunkBytes);
        for (int kc = 0; kc < nk; ++kc) {
            tma_load_2d(smem_u32(st.a_hi(kc, 0)), mhi, kc * KCH, i0, bar);
            tma_load_2d(smem_u32(st.a_hi(kc, 0) + kATileBytes), mlo, kc * KCH, i0, bar);
        }
    }
    const bool ok = mbar_wait(smem_u32(&b.res_full), st.nres & 1, st.status);
    st.nres += 1;
    __syncthreads();
    return ok;
}

// Tear-down: wait (bounded) for the last tile's MMAs, free TMEM.  All
// threads call it.
__device__ inline void tc_teardown(TcState& st) {
    TileBars& b = *st.bars;
    if (st.ntile > 0 && *((volatile int*)st.status) != 0)
        mbar_wait(smem_u32(&b.acc_full), (st.ntile - 1) & 1, st.status);
    if (st.wtile > 0 && *((volatile int*)st.status) != 0)
        mbar_wait(smem_u32(&b.wacc), (st.wtile - 1) & 1, st.status);
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    if ((threadIdx.x >> 5) == 0) tmem_dealloc(b.tmem_base, kTmemCols);
}

// Scale 2^e with |v| 2^e in [2^12, 2^13) for a vector of squared norm n2:
// with n2 in [2^k, 2^(k+1)), |v| is in [2^(k/2), 2^((k+1)/2)), so
// e = 12 - floor(k / 2), clamped to [-120, 120]; e = 0 for a zero, negative
// or non-finite n2.  Integer operations on the bits of n2 only.
__device__ __forceinline__ void vector_scale(double n2, float& scale, float& inv) {
    const long long bits = __double_as_longlong(n2);
    const int ex = (int)((bits >> 52) & 0x7ff);
    int e = 0;
    if (bits > 0 && ex != 0x7ff) {
        e = 12 - ((ex - 1023) >> 1);   // arithmetic shift: floor division by 2
        e = max(-120, min(120, e));
    }
    scale = __int_as_float((127 + e) << 23);
    inv = __int_as_float((127 - e) << 23);
}

// The same scale from an FP32 squared norm (exponent field of 8 bits).
__device__ __forceinline__ void vector_scale_f(float n2, float& scale, float& inv) {
    const int bits = __float_as_int(n2);
    const int ex = (bits >> 23) & 0xff;
    int e = 0;
    if (bits > 0 && ex != 0xff) {
        e = 12 - ((ex - 127) >> 1);
        e = max(-120, min(120, e));
    }
    scale = __int_as_float((127 + e) << 23);
    inv = __int_as_float((127 - e) << 23);
}

// One output tile: target slices t0 .. t0+ns-1 (ns <= NMAX/2), sites
// i0 .. i0+127.  Warp-specialised: warp 0 streams E_hi/E_lo chunks with TMA
// (streaming mode; in resident mode E is already in shared memory and warp 0
// only signals), warps 2..7 build the B chunks, warp 1 issues the MMAs as
// soon as a stage is full and releases it with tcgen05.commit.
// The epilogue runs on warps 4..7: Epi::load(i, t) fetches what the output
// (t, i) needs, Epi::store(i, t, in, w) receives w = (E u)_i for the tile's
// source slice of target t (unscaled; before shift sign and phase).
// Returns false if a bounded wait failed (status set).  All threads call it.
// res_b (streaming layout only): 0 builds B chunk by chunk in the ring;
// 1 first builds the B of all K chunks of slices t0..t0+ns-1 into the
// resident area with all threads, 2 reuses the resident B of the previous
// tile (same slices, another site block).  The epilogue runs on all eight
// warps once the roles are done (warps 4..7 the first half of the 16-column
// blocks, warps 0..3 the rest; a warp reads its TMEM lane quarter).
template <bool DAG, class Src, class Epi>
__device__ bool tc_tile(TcState& st, const CUtensorMap* mhi, const CUtensorMap* mlo, int V,
                        int Nt, int Vp, int i0, int t0, int ns, const Src& src, float scale,
                        float inv_scale, Epi& epi, int res_b = 0) {
    TileBars& bars = *st.bars;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nk = Vp / KCH;
    // MMA N: 2 x slices rounded up to 16; with B loaded by TMA, the box
    // height, so the expected bytes match the copy on a ragged last tile
    int N = ((2 * ns + 15) / 16) * 16;
    if constexpr (Src::kTma) N = src.rows;
    const int S = st.stages;
    const bool streaming = st.mode == kStreaming;
    const uint32_t g0 = st.gchunk;
    bool ok = true;
    const uint32_t chunk_b = (uint32_t)N * 128u;
    uint8_t* bres = st.base + st.b_off;
    if constexpr (!Src::kTma) {
        if (res_b == 1) {
            // all chunks of the tile's B at once: rows 2j (re), 2j+1 (im),
            // zero for slices >= ns and sites >= V
            const int nkb = Vp / 8;
            for (int w = threadIdx.x; w < (N / 2) * nkb; w += blockDim.x) {
                const int j = w / nkb, kbi = w - j * nkb, kb = kbi * 8;
                const int kc = kb / KCH, grp = kbi & 7;
                float2 v8[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) v8[e] = make_float2(0.f, 0.f);
                if (j < ns && kb < V) {
                    const int ts = source_slice<DAG>(t0 + j, Nt);
                    if (kb + 8 <= V) {
                        src.load8(ts, kb, v8);
                    } else {
#pragma unroll
                        for (int e = 0; e < 8; ++e)
                            if (kb + e < V) v8[e] = src.load1(ts, kb + e);
                    }
                }
                float re[8], im[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    re[e] = v8[e].x * scale;
                    im[e] = v8[e].y * scale;
                }
                uint4 hr, lr, hm, lm;
                split8(re, hr, lr);
                split8(im, hm, lm);
                const int jr = 2 * j, ji = jr + 1;
                uint8_t* bh = bres + (size_t)kc * chunk_b;
                uint8_t* bl = bh + (size_t)nk * chunk_b;
                *reinterpret_cast<uint4*>(bh + jr * 128 + ((grp ^ (jr & 7)) << 4)) = hr;
                *reinterpret_cast<uint4*>(bl + jr * 128 + ((grp ^ (jr & 7)) << 4)) = lr;
                *reinterpret_cast<uint4*>(bh + ji * 128 + ((grp ^ (ji & 7)) << 4)) = hm;
                *reinterpret_cast<uint4*>(bl + ji * 128 + ((grp ^ (ji & 7)) << 4)) = lm;
            }
            fence_proxy_async();
            __syncthreads();
        }
    }

    if (warp == kWarpTma) {
        if (lane == 0) {
            for (int kc = 0; kc < nk && ok; ++kc) {
                const uint32_t g = g0 + kc, s = g % S, n = g / S;
                if (n > 0) ok = mbar_wait(smem_u32(&bars.empty[s]), (n - 1) & 1, st.status);
                if (!ok) break;
                const uint32_t bar = smem_u32(&bars.full[s]);
                if constexpr (Src::kTma) {
                    // streaming layout only: E and the pre-split B of chunk kc
                    mbar_arrive_expect_tx(bar, kAChunkBytes + 2u * (uint32_t)N * 128u);
                    tma_load_2d(smem_u32(st.a_hi(kc, s)), mhi, kc * KCH, i0, bar);
                    tma_load_2d(smem_u32(st.a_hi(kc, s) + kATileBytes), mlo, kc * KCH, i0, bar);
                    tma_load_2d(smem_u32(st.b_hi(s)), src.bhi, kc * KCH, 2 * t0, bar);
                    tma_load_2d(smem_u32(st.b_hi(s)) + st.b_stage / 2, src.blo, kc * KCH, 2 * t0,
                                bar);
                } else if (streaming) {
                    mbar_arrive_expect_tx(bar, kAChunkBytes);
                    tma_load_2d(smem_u32(st.a_hi(kc, s)), mhi, kc * KCH, i0, bar);
                    tma_load_2d(smem_u32(st.a_hi(kc, s) + kATileBytes), mlo, kc * KCH, i0, bar);
                } else {
                    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar)
                                 : "memory");
                }
            }
        }
    } else if (warp == kWarpMma) {
        if (lane == 0) {
            const uint32_t idesc = idesc_f16(TM, N);
            const uint32_t tmem = bars.tmem_base;
            for (int kc = 0; kc < nk && ok; ++kc) {
                const uint32_t g = g0 + kc, s = g % S, n = g / S;
                ok = mbar_wait(smem_u32(&bars.full[s]), n & 1, st.status);
                if (!ok) break;
                fence_after_sync();
                const uint32_t ah = smem_u32(st.a_hi(kc, s)), al = ah + kATileBytes;
                uint32_t bh = smem_u32(st.b_hi(s)), bl = bh + st.b_stage / 2;
                if (res_b != 0) {
                    bh = smem_u32(bres + (size_t)kc * chunk_b);
                    bl = bh + (uint32_t)nk * chunk_b;
                }
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
                mma_commit(smem_u32(&bars.empty[s]));
            }
            mma_commit(smem_u32(&bars.acc_full));
        }
    } else {
        // B producers (warps 2..7).  A chunk has (N/2)*8 items; when one
        // group of producer warps can hold a chunk at one item per thread,
        // the six warps split into groups that build successive chunks at
        // the same time (chunk kc goes to group kc % groups).  Every warp
        // still waits for each chunk's stage and arrives on its full barrier
        // (warps of other groups without writing), so the arrival count is
        // the same for every chunk and no arrival can precede the stage's
        // release.
        const int pw = warp - kFirstBWarp;
        const int items = (N >> 1) * 8;
        const int groups = items <= 128 ? 3 : (items <= 192 ? 2 : 1);
        const int gw = kNumBWarps / groups;              // warps per group
        const int my_group = pw / gw;
        const int ptid = (pw % gw) * 32 + lane, nprod = gw * 32;
        for (int kc = 0; kc < nk && ok; ++kc) {
            const uint32_t g = g0 + kc, s = g % S, n = g / S;
            if (n > 0) ok = mbar_wait(smem_u32(&bars.empty[s]), (n - 1) & 1, st.status);
            if (!ok) break;
            if constexpr (!Src::kTma) {
                if (res_b == 0 && kc % groups == my_group) {
                    uint8_t* bh = st.b_hi(s);
                    build_B<DAG>(src, V, Nt, t0, ns, N, kc * KCH, scale, bh, bh + st.b_stage / 2,
                                 ptid, nprod);
                    fence_proxy_async();
                }
            }
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(
                                            smem_u32(&bars.full[s]))
                                        : "memory");
        }
    }
    // epilogue on all warps: lane quarter (warp % 4) of TMEM, 16-column
    // blocks [b0, b1).  The inputs of a block of 8 slices are fetched
    // together (the first block before the accumulator is ready, overlapping
    // the MMA tail).
    __syncwarp();
    {
        const int nb = N / 16, half = (nb + 1) / 2;
        const bool hi_warps = warp >= kFirstEpiWarp;
        const int b0 = hi_warps ? 0 : half, b1 = hi_warps ? half : nb;
        using In = typename Epi::In;
        const int row = (warp & 3) * 32 + lane;
        const int i = i0 + row;
        In cur[8];
        auto fetch = [&](int cb, In (&dst)[8]) {
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int tt = (cb >> 1) + e;
                if (i < V && tt < ns) dst[e] = epi.load(i, t0 + tt);
            }
        };
        if (b0 < b1) {
            if (ok) fetch(b0 * 16, cur);
            if (ok) ok = mbar_wait(smem_u32(&bars.acc_full), st.ntile & 1, st.status);
            fence_after_sync();
            ok = __all_sync(0xffffffffu, ok);   // tcgen05.ld below is warp-collective
            if (ok) {
                const uint32_t tl = bars.tmem_base + ((uint32_t)((warp & 3) * 32) << 16);
                for (int cb = b0 * 16; cb < b1 * 16; cb += 16) {
                    if (cb > b0 * 16) fetch(cb, cur);
                    float m[16], c[16];
                    tmem_ld16(tl + cb, m);
                    tmem_ld16(tl + kCorrCol + cb, c);
#pragma unroll
                    for (int e = 0; e < 8; ++e) {
                        const int tt = (cb >> 1) + e;
                        if (i < V && tt < ns) {
                            float is = inv_scale;
                            if constexpr (Src::kTma) is = src.inv[t0 + tt];
                            const float wr = fmaf(c[2 * e], kLoInv, m[2 * e]) * is;
                            const float wi = fmaf(c[2 * e + 1], kLoInv, m[2 * e + 1]) * is;
                            epi.store(i, t0 + tt, cur[e], make_float2(wr, wi));
                        }
                    }
                }
            }
        }
    }
    st.gchunk = g0 + nk;
    st.ntile += 1;
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    return *((volatile int*)st.status) == 0;
}

}  // namespace tc
}  // namespace hmc
