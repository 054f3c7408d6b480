// tc_kernels.cu -- the mixed-precision path: tensor-core applications of
// M / M^dag (FP16 split, FP32 accumulate), FP32 conjugate gradient with FP64
// reliable updates, and the HMC trajectory built on it.  FP64 stays for the
// true residual, chi = M rho, the force, the Hamiltonian sums and Metropolis.
#include <cuda_fp16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "fp64_path.cuh"
#include "tc_path.h"
#include "tc_tile.cuh"
#include "tc_wide.cuh"
#include "tc_splitk.cuh"
#include "small_cg.cuh"

namespace hmc {

struct TcCtx {
    CUtensorMap map_hi, map_lo;
    int ns_apply;        // slices per tile of standalone applications
    // pre-split B operand of standalone applications: FP16 hi / lo rows
    // [2 Nt + 64][Vp] (row 2t: re, 2t+1: im of the source of target slice t;
    // the last 64 rows stay zero for tiles that run past Nt) and the
    // per-slice inverse scales
    CUtensorMap map_bhi, map_blo;
    __half* bhi;
    __half* blo;
    float* inv_col;
    int b_rows;
    // slice-major tiles (operand_mode 4): maps of the scaled split of E (box
    // rows = W / nmma), sites per tile of the solver and of standalone
    // applications, slices per standalone tile, and the maps of the
    // pre-split U (plain remainder) over bhi / blo with 128-row boxes
    CUtensorMap map_whi, map_wlo, map_uhi, map_ulo;
    int w_cg, w_apply, ns_wapply, csplit_apply;
    // split-K tiles (operand_mode 5): the scaled split of E in 128-row boxes;
    // standalone applications: the shape (C CTAs per cluster, ns slices per
    // n-group, 0 if it does not fit) and the maps of the pre-split source
    // (plain remainder) over bhi / blo with boxes of sk_nn(ns) rows
    CUtensorMap map_shi, map_slo;
    int sk_C_apply, sk_ns_apply;
    float* inv_sk;       // per (target slice, K range) inverse scales [Nt][C]
    CUtensorMap map_skb_hi, map_skb_lo;
};

namespace tc {
// TMA box rows of the pre-split U for tiles of ns slices: 2 ns rounded up
// to 16 (the swizzle atom is 8 rows; whole 1024-byte atoms), at most 128.
__host__ __device__ inline int wide_u_rows(int ns) {
    const int r = ((2 * ns + 15) / 16) * 16;
    return r > 128 ? 128 : r;
}
}  // namespace tc

namespace tc {

// ---------------------------------------------------------------- epilogues
// Each epilogue splits into load (global reads of what output (t, i) needs)
// and store (arithmetic and writes), so the tile can batch the reads.
template <bool DAG>
struct EpiStore {
    const float2* in;
    float2* out;
    const float2* cis;
    int V, Nt;
    float acc;   // per-thread partial |out|^2 (at most 32 terms; FP32 suffices)
    struct In {
        float2 s, ph;
    };
    __device__ __forceinline__ In load(int i, int t) const {
        const size_t o = (size_t)t * V + i;
        In v;
        v.s = in[o];
        v.ph = DAG ? cis[o] : make_float2(1.f, 0.f);
        return v;
    }
    __device__ __forceinline__ void store(int i, int t, const In& v, float2 w) {
        float sg;
        if (DAG) {
            sg = (t == Nt - 1) ? -1.f : 1.f;
            w = cmulcf(v.ph, w);
        } else {
            sg = (t == 0) ? -1.f : 1.f;
        }
        const float2 r = make_float2(v.s.x - sg * w.x, v.s.y - sg * w.y);
        out[(size_t)t * V + i] = r;
        acc = fmaf(r.x, r.x, fmaf(r.y, r.y, acc));
    }
    // sites i, i+1 (i even) with 16-byte accesses
    struct In2 {
        float4 s, ph;
    };
    __device__ __forceinline__ In2 load2(int i, int t) const {
        const size_t o = (size_t)t * V + i;
        In2 v;
        v.s = *reinterpret_cast<const float4*>(in + o);
        v.ph = DAG ? *reinterpret_cast<const float4*>(cis + o) : make_float4(1.f, 0.f, 1.f, 0.f);
        return v;
    }
    __device__ __forceinline__ void store2(int i, int t, const In2& v, float2 w0, float2 w1) {
        float sg;
        if (DAG) {
            sg = (t == Nt - 1) ? -1.f : 1.f;
            w0 = cmulcf(make_float2(v.ph.x, v.ph.y), w0);
            w1 = cmulcf(make_float2(v.ph.z, v.ph.w), w1);
        } else {
            sg = (t == 0) ? -1.f : 1.f;
        }
        const float4 r = make_float4(v.s.x - sg * w0.x, v.s.y - sg * w0.y, v.s.z - sg * w1.x,
                                     v.s.w - sg * w1.y);
        *reinterpret_cast<float4*>(out + (size_t)t * V + i) = r;
        acc = fmaf(r.x, r.x, fmaf(r.y, r.y, acc));
        acc = fmaf(r.z, r.z, fmaf(r.w, r.w, acc));
    }
};

// M q -> Ap; x_f += alpha p; r_f -= alpha Ap; accumulates |r_f|^2.
struct EpiCgUpdate {
    const float2* q;
    const float2* p;
    float2* x;
    float2* r;
    float alpha;
    int V;
    float acc;   // per-thread partial |r|^2
    struct In {
        float2 q, p, x, r;
    };
    __device__ __forceinline__ In load(int i, int t) const {
        const size_t o = (size_t)t * V + i;
        In v;
        v.q = q[o];
        v.p = p[o];
        v.x = x[o];
        v.r = r[o];
        return v;
    }
    __device__ __forceinline__ void store(int i, int t, const In& v, float2 w) {
        const size_t o = (size_t)t * V + i;
        const float sg = (t == 0) ? -1.f : 1.f;
        const float2 ap = make_float2(v.q.x - sg * w.x, v.q.y - sg * w.y);
        float2 xv = v.x, rv = v.r;
        xv.x = fmaf(alpha, v.p.x, xv.x);
        xv.y = fmaf(alpha, v.p.y, xv.y);
        rv.x = fmaf(-alpha, ap.x, rv.x);
        rv.y = fmaf(-alpha, ap.y, rv.y);
        x[o] = xv;
        r[o] = rv;
        acc = fmaf(rv.x, rv.x, fmaf(rv.y, rv.y, acc));
    }
    struct In2 {
        float4 q, p, x, r;
    };
    __device__ __forceinline__ In2 load2(int i, int t) const {
        const size_t o = (size_t)t * V + i;
        In2 v;
        v.q = *reinterpret_cast<const float4*>(q + o);
        v.p = *reinterpret_cast<const float4*>(p + o);
        v.x = *reinterpret_cast<const float4*>(x + o);
        v.r = *reinterpret_cast<const float4*>(r + o);
        return v;
    }
    __device__ __forceinline__ void store2(int i, int t, const In2& v, float2 w0, float2 w1) {
        const size_t o = (size_t)t * V + i;
        const float sg = (t == 0) ? -1.f : 1.f;
        const float4 ap = make_float4(v.q.x - sg * w0.x, v.q.y - sg * w0.y, v.q.z - sg * w1.x,
                                      v.q.w - sg * w1.y);
        const float4 xv = make_float4(fmaf(alpha, v.p.x, v.x.x), fmaf(alpha, v.p.y, v.x.y),
                                      fmaf(alpha, v.p.z, v.x.z), fmaf(alpha, v.p.w, v.x.w));
        const float4 rv = make_float4(fmaf(-alpha, ap.x, v.r.x), fmaf(-alpha, ap.y, v.r.y),
                                      fmaf(-alpha, ap.z, v.r.z), fmaf(-alpha, ap.w, v.r.w));
        *reinterpret_cast<float4*>(x + o) = xv;
        *reinterpret_cast<float4*>(r + o) = rv;
        acc = fmaf(rv.x, rv.x, fmaf(rv.y, rv.y, acc));
        acc = fmaf(rv.z, rv.z, fmaf(rv.w, rv.w, acc));
    }
};

// CG direction step fused into M^dag: at the tile's own (t, i) form
// p_new = r + beta p_old (r from the FP64 residual after a reliable update,
// which is then also stored as the new FP32 r), store p_new, and
// q = M^dag p_new = p_new - s_{t+1} e^{-i phi_t} w; accumulates |q|^2.
struct EpiDirection {
    SrcDirection d;
    float2* p_new;
    float2* r_out;     // written when d.refresh
    float2* q;
    const float2* cis;
    int Nt;
    float acc;   // per-thread partial |q|^2
    struct In {
        float2 r, p, ph;
    };
    __device__ __forceinline__ In load(int i, int t) const {
        const size_t o = (size_t)t * d.V + i;
        In v;
        if (d.refresh) {
            const double2 r64 = d.r64[o];
            v.r = make_float2((float)r64.x, (float)r64.y);
        } else {
            v.r = d.r[o];
        }
        v.p = d.p_old[o];
        v.ph = cis[o];
        return v;
    }
    __device__ __forceinline__ void store(int i, int t, const In& v, float2 w) {
        const size_t o = (size_t)t * d.V + i;
        const float2 pv = make_float2(fmaf(d.beta, v.p.x, v.r.x), fmaf(d.beta, v.p.y, v.r.y));
        if (d.refresh) r_out[o] = v.r;
        p_new[o] = pv;
        const float sg = (t == Nt - 1) ? -1.f : 1.f;
        w = cmulcf(v.ph, w);
        const float2 qv = make_float2(pv.x - sg * w.x, pv.y - sg * w.y);
        q[o] = qv;
        acc = fmaf(qv.x, qv.x, fmaf(qv.y, qv.y, acc));
    }
    struct In2 {
        float4 r, p, ph;
    };
    __device__ __forceinline__ In2 load2(int i, int t) const {
        const size_t o = (size_t)t * d.V + i;
        In2 v;
        if (d.refresh) {
            const double2 a = d.r64[o], b = d.r64[o + 1];
            v.r = make_float4((float)a.x, (float)a.y, (float)b.x, (float)b.y);
        } else {
            v.r = *reinterpret_cast<const float4*>(d.r + o);
        }
        v.p = *reinterpret_cast<const float4*>(d.p_old + o);
        v.ph = *reinterpret_cast<const float4*>(cis + o);
        return v;
    }
    __device__ __forceinline__ void store2(int i, int t, const In2& v, float2 w0, float2 w1) {
        const size_t o = (size_t)t * d.V + i;
        const float4 pv = make_float4(fmaf(d.beta, v.p.x, v.r.x), fmaf(d.beta, v.p.y, v.r.y),
                                      fmaf(d.beta, v.p.z, v.r.z), fmaf(d.beta, v.p.w, v.r.w));
        if (d.refresh) *reinterpret_cast<float4*>(r_out + o) = v.r;
        *reinterpret_cast<float4*>(p_new + o) = pv;
        const float sg = (t == Nt - 1) ? -1.f : 1.f;
        w0 = cmulcf(make_float2(v.ph.x, v.ph.y), w0);
        w1 = cmulcf(make_float2(v.ph.z, v.ph.w), w1);
        const float4 qv = make_float4(pv.x - sg * w0.x, pv.y - sg * w0.y, pv.z - sg * w1.x,
                                      pv.w - sg * w1.y);
        *reinterpret_cast<float4*>(q + o) = qv;
        acc = fmaf(qv.x, qv.x, fmaf(qv.y, qv.y, acc));
        acc = fmaf(qv.z, qv.z, fmaf(qv.w, qv.w, acc));
    }
};

__device__ __forceinline__ void tile_coords(int tile, int nti, int ns_tile, int Nt, int& i0,
                                            int& t0, int& ns) {
    i0 = (tile % nti) * TM;
    t0 = (tile / nti) * ns_tile;
    ns = min(ns_tile, Nt - t0);
}

// All tensor-core tiles of one application, spread over the team.
template <bool DAG, class Src, class Epi>
__device__ bool apply_team(const ChainView& c, const Team& tm, TcState& st,
                           const CUtensorMap* mhi, const CUtensorMap* mlo, int ns_tile,
                           const Src& src, float scale, float inv, Epi& epi,
                           bool res_b = false) {
    const int nti = c.Vr / TM, ntt = (c.Nt + ns_tile - 1) / ns_tile;
    // tiles are dealt round robin over the team; in resident mode the team
    // size is a multiple of the site blocks, so a CTA only meets tiles of
    // its own site block (rank mod nti), whose rows of E it holds.  With a
    // resident B, slice tiles go round robin and a CTA runs all site blocks
    // of each of its slice tiles, building that B once.  One call site of
    // the tile keeps it inlined once.
    for (int j = 0;; ++j) {
        int i0, t0, ns, rflag = 0;
        if (res_b) {
            const int stl = tm.rank + (j / nti) * tm.size, rb = j % nti;
            if (stl >= ntt) break;
            i0 = rb * TM;
            t0 = stl * ns_tile;
            ns = min(ns_tile, c.Nt - t0);
            rflag = rb == 0 ? 1 : 2;
        } else {
            const int tile = tm.rank + j * tm.size;
            if (tile >= nti * ntt) break;
            tile_coords(tile, nti, ns_tile, c.Nt, i0, t0, ns);
        }
        if (!tc_tile<DAG>(st, mhi, mlo, c.V, c.Nt, c.Vp, i0, t0, ns, src, scale, inv, epi, rflag))
            return false;
    }
    return true;
}

// All slice-major tiles of one application (W sites x ns_tile slices each),
// dealt round robin over the team.
template <bool DAG, class Src, class Epi>
__device__ bool apply_team_w(const ChainView& c, const Team& tm, TcState& st, int W,
                             const CUtensorMap* mhi, const CUtensorMap* mlo, int ns_tile,
                             const Src& src, float scale, float inv, Epi& epi) {
    const WideGeom g = wide_geom(W);
    const int nsi = (c.V + W - 1) / W, ntt = (c.Nt + ns_tile - 1) / ns_tile;
    for (int tile = tm.rank; tile < nsi * ntt; tile += tm.size) {
        const int i0 = (tile % nsi) * W, t0 = (tile / nsi) * ns_tile;
        const int ns = min(ns_tile, c.Nt - t0);
        if (!tc_wtile<DAG>(st, g, mhi, mlo, c.V, c.Nt, c.Vp, i0, t0, ns, src, scale, inv,
                           c.e_inv, epi))
            return false;
    }
    return true;
}

// ---------------------------------------------------------------- standalone
// B operand of one standalone application, split before the tiles run: for
// target slice t (one block) the source u = in_{t+1} (M^dag) or
// e^{i phi_{t-1}} in_{t-1} (M), scaled by 2^e with max |Re u|, |Im u| in
// [2^14, 2^15), written as FP16 hi = fp16(s u) and lo = fp16((s u - hi) 2^11)
// (PLAIN, for the slice-major tile: lo = fp16(s u - hi)) in rows 2t (re) and
// 2t+1 (im), zero from V to Vp; inv[t] = 2^-e.  Also writes the FP32 phase
// table of slice t (the M^dag epilogue reads it).
// Dynamic shared memory: V float2 (the source slice).  1024 threads per
// block: the work per slice is a few sites per thread, so the block's two
// passes are each about one round trip to memory.
constexpr int kSplitThreads = 1024;
template <bool DAG, bool PLAIN>
__global__ void __launch_bounds__(kSplitThreads)
    k_split(const double* __restrict__ phi, const float2* __restrict__ in,
            float2* __restrict__ cis_f, __half* __restrict__ bhi, __half* __restrict__ blo,
            float* __restrict__ inv, int V, int Vp, int Nt) {
    extern __shared__ float2 u_s[];
    __shared__ float s_max[kSplitThreads / 32];
    __shared__ int s_e;
    // the application kernel may start its set-up now (programmatic
    // dependent launch); it waits for this grid before reading B
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const int t = blockIdx.x;
    const int ts = DAG ? (t + 1 == Nt ? 0 : t + 1) : (t == 0 ? Nt - 1 : t - 1);
    float mx = 0.f;
    for (int k = threadIdx.x; k < V; k += blockDim.x) {
        float sn, cs;
        sincosf((float)phi[(size_t)t * V + k], &sn, &cs);
        cis_f[(size_t)t * V + k] = make_float2(cs, sn);
        float2 u = in[(size_t)ts * V + k];
        if (!DAG) {
            sincosf((float)phi[(size_t)ts * V + k], &sn, &cs);
            u = make_float2(cs * u.x - sn * u.y, cs * u.y + sn * u.x);
        }
        u_s[k] = u;
        mx = fmaxf(mx, fmaxf(fabsf(u.x), fabsf(u.y)));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_down_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) s_max[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        float m = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, s_max[w]);
        const int bits = __float_as_int(m), ex = (bits >> 23) & 0xff;
        int e = 0;
        if (bits > 0 && ex != 0xff) e = max(-120, min(120, 14 - (ex - 127)));
        s_e = e;
        inv[t] = __int_as_float((127 - e) << 23);
    }
    __syncthreads();
    const float sc = __int_as_float((127 + s_e) << 23);
    __half* hr = bhi + (size_t)(2 * t) * Vp;
    __half* lr = blo + (size_t)(2 * t) * Vp;
    for (int k = threadIdx.x; k < Vp; k += blockDim.x) {
        __half h0 = __float2half_rn(0.f), h1 = h0, l0 = h0, l1 = h0;
        if (k < V) {
            const float2 u = u_s[k];
            const float x = u.x * sc, y = u.y * sc;
            h0 = __float2half_rn(x);
            h1 = __float2half_rn(y);
            const float ls = PLAIN ? 1.f : kLoScale;
            l0 = __float2half_rn((x - __half2float(h0)) * ls);
            l1 = __float2half_rn((y - __half2float(h1)) * ls);
        }
        hr[k] = h0;
        hr[Vp + k] = h1;
        lr[k] = l0;
        lr[Vp + k] = l1;
    }
}

// Standalone application of M or M^dag: the tiles load E and the pre-split
// B by TMA and contract them; the epilogue forms the result.
template <bool DAG>
__global__ void __launch_bounds__(NTHR, 1)
    k_apply(const __grid_constant__ CUtensorMap mhi, const __grid_constant__ CUtensorMap mlo,
            const __grid_constant__ CUtensorMap bhi, const __grid_constant__ CUtensorMap blo,
            ChainView c, int ns_tile, const float2* in, float2* out, const float* inv) {
    extern __shared__ __align__(1024) uint8_t dyn[];
    TcState st;
    tc_setup(st, dyn, c.status);
    EpiStore<DAG> epi{in, out, c.cis_f, c.V, c.Nt, 0.f};
    const int nti = c.Vr / TM;
    int i0, t0, ns;
    tile_coords(blockIdx.x, nti, ns_tile, c.Nt, i0, t0, ns);
    SrcSplit src{&bhi, &blo, inv, ((2 * ns_tile + 15) / 16) * 16};
    // launched as a programmatic dependent of the split: the set-up above
    // overlaps it; its B, scales and phase table are visible after this
    asm volatile("griddepcontrol.wait;" ::: "memory");
    tc_tile<DAG>(st, &mhi, &mlo, c.V, c.Nt, c.Vp, i0, t0, ns, src, 1.f, 1.f, epi);
    tc_teardown(st);
}

// Standalone application on slice-major tiles: one output tile (W sites x
// ns_tile slices) per thread-block cluster of csplit CTAs, which split its K
// chunks; E' and the pre-split U arrive by TMA.  Each CTA contracts its
// chunks into its own accumulator and stages it in shared memory; after a
// cluster barrier each takes a share of the tile's outputs, sums the csplit
// partials through distributed shared memory in rank order and runs the
// epilogue; a second cluster barrier keeps every CTA's shared memory alive
// until the others have read it.  csplit = 1 is a plain launch.
template <bool DAG>
__global__ void __launch_bounds__(NTHR, 1)
    k_apply_w(const __grid_constant__ CUtensorMap mhi, const __grid_constant__ CUtensorMap mlo,
              const __grid_constant__ CUtensorMap uhi, const __grid_constant__ CUtensorMap ulo,
              ChainView c, int W, int ns_tile, int csplit, const float2* in, float2* out,
              const float* inv) {
    extern __shared__ __align__(1024) uint8_t dyn[];
    TcState st;
    tc_setup(st, dyn, c.status);
    EpiStore<DAG> epi{in, out, c.cis_f, c.V, c.Nt, 0.f};
    const WideGeom g = wide_geom(W);
    const int nsi = (c.V + W - 1) / W, nk = c.Vp / KCH;
    const int tile = blockIdx.x / csplit, rank = blockIdx.x % csplit;
    const int i0 = (tile % nsi) * W, t0 = (tile / nsi) * ns_tile;
    const int ns = min(ns_tile, c.Nt - t0);
    const int kc0 = nk * rank / csplit, kc1 = nk * (rank + 1) / csplit;
    SrcSplitW src{&uhi, &ulo, inv, wide_u_rows(ns_tile)};
    asm volatile("griddepcontrol.wait;" ::: "memory");   // the split (see k_apply)
    tc_wstage<DAG>(st, g, &mhi, &mlo, c.V, c.Nt, i0, t0, ns, kc0, kc1, src, 1.f);
    cluster_barrier_all();   // every member's partial staged (release / acquire)
    if (*((volatile int*)c.status) == 0)
        tc_wepilogue(st, W, c.V, i0, t0, ns, src, 1.f, c.e_inv, epi, rank, csplit);
    cluster_barrier_all();   // the partials stay until every member has read them
    tc_teardown(st);
}

// B operand of a standalone split-K application, one block per (target
// slice t, K range r of the clusters' C CTAs): the source u of slice t
// (in_{t+1} for M^dag, e^{i phi_{t-1}} in_{t-1} for M) over the range's
// sites, scaled by 2^e with the largest |Re u|, |Im u| of the range in
// [2^14, 2^15), split into FP16 hi and plain remainder lo in rows 2t (re)
// and 2t + 1 (im); inv[t * C + r] = 2^-e (the consumer unscales its
// partial per column with it: the scale is uniform over its K range).  Also
// the FP32 phase table of slice t over the range.  One element per thread;
// one pass over memory.
constexpr int kSplitSkThreads = 256;   // >= the largest K range (4 chunks of 64)
template <bool DAG>
__global__ void __launch_bounds__(kSplitSkThreads)
    k_split_sk(const double* __restrict__ phi, const float2* __restrict__ in,
               float2* __restrict__ cis_f, __half* __restrict__ bhi, __half* __restrict__ blo,
               float* __restrict__ inv, int V, int Vp, int Nt, int C) {
    __shared__ float s_max[kSplitSkThreads / 32];
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const int t = blockIdx.x, r = blockIdx.y;
    const int KS = (V + 15) / 16;
    const int k0 = 16 * (KS * r / C), k1 = min(16 * (KS * (r + 1) / C), V);
    const int ts = DAG ? (t + 1 == Nt ? 0 : t + 1) : (t == 0 ? Nt - 1 : t - 1);
    const int k = k0 + (int)threadIdx.x;
    float2 u = make_float2(0.f, 0.f);
    if (k < k1) {
        float sn, cs;
        sincosf((float)phi[(size_t)t * V + k], &sn, &cs);
        cis_f[(size_t)t * V + k] = make_float2(cs, sn);
        u = in[(size_t)ts * V + k];
        if (!DAG) {
            sincosf((float)phi[(size_t)ts * V + k], &sn, &cs);
            u = make_float2(cs * u.x - sn * u.y, cs * u.y + sn * u.x);
        }
    }
    float mx = fmaxf(fabsf(u.x), fabsf(u.y));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) s_max[threadIdx.x >> 5] = mx;
    __syncthreads();
    float m = 0.f;
    for (int w = 0; w < kSplitSkThreads / 32; ++w) m = fmaxf(m, s_max[w]);
    const int bits = __float_as_int(m), ex = (bits >> 23) & 0xff;
    int e = 0;
    if (bits > 0 && ex != 0xff) e = max(-120, min(120, 14 - (ex - 127)));
    if (threadIdx.x == 0) inv[t * C + r] = __int_as_float((127 - e) << 23);
    if (k < k1) {
        const float sc = __int_as_float((127 + e) << 23);
        const float x = u.x * sc, y = u.y * sc;
        const __half h0 = __float2half_rn(x), h1 = __float2half_rn(y);
        bhi[(size_t)(2 * t) * Vp + k] = h0;
        bhi[(size_t)(2 * t + 1) * Vp + k] = h1;
        blo[(size_t)(2 * t) * Vp + k] = __float2half_rn(x - __half2float(h0));
        blo[(size_t)(2 * t + 1) * Vp + k] = __float2half_rn(y - __half2float(h1));
    }
}

// Standalone application on split-K tiles (operand_mode 5): clusters of C
// CTAs, cluster (ib, ng) = site block ib x n-group ng of ns target slices;
// each CTA loads its 128 rows x K range of the scaled split of E by TMA
// (before waiting for the split pre-pass, which it does not read), then the
// pre-split source rows 2 t0 .. 2 t0 + Nn of its K range (plain FP16 hi and
// lo, one power-of-two scale per target slice and K range), one barrier per
// 64-wide K chunk, and issues each chunk's MMAs as it lands; it stages its
// partial unscaled per column by its own range's scales.  The C partials of a
// cluster are summed through distributed shared memory in rank order by the
// owners of the outputs (deterministic); a last cluster barrier keeps every
// member's shared memory alive until the others have read it.  E moves
// from L2 once per application (not once per slice tile).
template <bool DAG>
__global__ void __launch_bounds__(NTHR, 1)
    k_apply_sk(const __grid_constant__ CUtensorMap mhi, const __grid_constant__ CUtensorMap mlo,
               const __grid_constant__ CUtensorMap bhi, const __grid_constant__ CUtensorMap blo,
               ChainView c, int C, int ns, const float2* in, float2* out, const float* inv) {
    extern __shared__ __align__(1024) uint8_t dyn[];
    TcState st;
    tc_setup(st, dyn, c.status);
    const SkGeom g = sk_geom(blockIdx.x, C, ns, c.V, c.Nt, c.Vr, c.Vp);
    TileBars& b = *st.bars;
    const uint32_t cb = 2u * (uint32_t)g.Nn * 128u;   // bytes of one stacked B chunk
    if (threadIdx.x == 0) {
        const uint32_t bar = smem_u32(&b.res_full);
        mbar_arrive_expect_tx(bar, (uint32_t)g.nch * kAChunkBytes);
        for (int j = 0; j < g.nch; ++j) {
            const uint32_t dst = smem_u32(st.base + (size_t)j * kAChunkBytes);
            const int x = 16 * g.ks0 + KCH * j;   // a multiple of 16 elements
            tma_load_2d(dst, &mhi, x, g.ib * TM, bar);
            tma_load_2d(dst + kATileBytes, &mlo, x, g.ib * TM, bar);
        }
    }
    // launched as a programmatic dependent of the split (see k_apply)
    asm volatile("griddepcontrol.wait;" ::: "memory");
    if (threadIdx.x == 0) {
        for (int j = 0; j < g.nch; ++j) {
            const uint32_t bar = smem_u32(&b.skb[j]);
            const uint32_t dst = smem_u32(st.base + g.b_off + (size_t)j * cb);
            const int x = 16 * g.ks0 + KCH * j;
            mbar_arrive_expect_tx(bar, cb);
            tma_load_2d(dst, &bhi, x, 2 * g.t0, bar);
            tma_load_2d(dst + (uint32_t)g.Nn * 128u, &blo, x, 2 * g.t0, bar);
        }
        bool ok = mbar_wait(smem_u32(&b.res_full), 0, st.status);
        for (int j = 0; j < g.nch && ok; ++j) {
            ok = mbar_wait(smem_u32(&b.skb[j]), 0, st.status);
            if (ok) sk_issue_chunk(st, g, j, smem_u32(st.base + g.b_off + (size_t)j * cb),
                                   b.tmem_base);
        }
    }
    Team none = {};
    SkEpiOut<DAG> epi{in, out, c.cis_f, c.V, c.Nt};
    sk_finish<true>(st, g, none, c.V, c.e_inv, epi, inv, c.Nt);
    cluster_barrier_all();   // the partials stay until every member has read them
    tc_teardown(st);
}

// ---------------------------------------------------------------- mixed CG
struct MixedResult {
    int iterations;
    int reliable_updates;
    double true_res;
    int status;
    int fp64_iterations;   // iterations of the FP64 fallback (0 if it did not run)
};

struct PersistentArgs {
    int ns_tile;
    int inner;         // CTAs of the FP32 inner loop
    int cluster;       // > 1: launched in clusters of this size, the inner team is cluster 0
    int res_b;         // streaming layout: resident B per slice tile (apply_team)
    int mode;          // OperandMode: resident needs inner a multiple of the site blocks
    int wide_W;        // kSlice: sites per slice-major tile
    int vec_resident;  // resident mode with one CTA: FP32 CG vectors in shared memory
    double tol;
    int max_iter;
    double ru_delta;
    int ru_every;      // reliable update after this many FP32 iterations at the latest
    int sk_C;          // kSplitK: CTAs per cluster splitting K (ns_tile: slices per n-group)
};

struct BatchItem {
    ChainView v;
    int team;                  // > 1: run by a cluster of this many CTAs (the launch's size)
    const CUtensorMap* maps;   // [0] E_hi, [1] E_lo, [2] / [3] scaled split for the
                               // slice-major tile (global memory, 64-byte aligned)
    PersistentArgs pa;
    TrajArgs a;                // n_md, eps, tol, max_iter, chain; seed/traj/phi per call
    long long offset;          // of this chain's field in the packed array
};

struct BatchCallArgs {
    uint64_t seed;
    uint64_t traj;
    double* phi;               // packed fields of all chains
};

// FP64 true residual of x64: r64 = chi - M (M^dag x64); returns |r64|^2.
__device__ bool f64_residual(const ChainView& c, Team& tm, f64::Smem& sm, const double2* chi,
                             double2* x64, double& rr, double gm1 = 0.0) {
    f64::EpiArgs ea = {};
    ea.hop_m1 = gm1;   // M_g = 1 - g S E D with g = 1 + gm1 (mass preconditioning)
    f64::apply_team<true, f64::EPI_STORE>(c, tm, x64, c.q, ea, sm);
    if (!team_barrier(tm)) return false;
    ea.chi = chi;
    ea.r = c.r;
    double v[1] = {f64::apply_team<false, f64::EPI_RESIDUAL>(c, tm, c.q, nullptr, ea, sm)};
    if (!team_sum<1>(tm, v)) return false;
    rr = v[0];
    return true;
}

// FP32 CG on the tensor-core operator with FP64 reliable updates
// (Sleijpen-van der Vorst style, as used in lattice QCD solvers): whenever
// the iterated residual has dropped by ru_delta since the last update, or
// claims convergence, the FP32 increment is folded into the FP64 solution,
// the true residual chi - M M^dag x is recomputed in FP64 and replaces the
// iterated one; the search direction is kept.  Stops on the FP64 true
// residual.
//
// Two teams: the FP32 iterations run on the first `inner` CTAs (one CTA
// for small lattices, so an iteration needs no inter-CTA barrier), the FP64
// steps on all CTAs of the launch (FP64 is ~1/1700 of the tensor rate, so it
// is spread over as many SMs as possible).  The other CTAs wait at the
// outer barrier while the inner loop runs.  Two inner synchronisations per
// iteration: the direction update p = r + beta p happens inside the M^dag
// application (operand build and epilogue, into a second p buffer), the
// x / r update inside the M one.  Needs c.cis and c.cis_f of the current phi.
enum SegmentEnd : int { kSegUpdate = 1, kSegMaxIter = 2, kSegNonfinite = 3 };

// Scalar state of the FP32 iteration, kept and updated by thread 0 alone
// and read by the other threads after a barrier, in FP32 (the iterates are
// FP32; FP64 arithmetic runs at a small fraction of the FP32 rate and with
// long latency on this part).  rr = |r|^2, pp = |p|^2 estimate (sets the
// vector scale of the tensor-core operands), rmax = |r|^2 at the last
// reliable update; stop and ru2 are the FP32 images of the FP64 criteria.
struct CgScalars {
    float rr, pp, rmax, alpha, beta, sc, inv, stop, ru2;
    int it, reason;
    int it0, every;   // iteration of the last reliable update; the most between two
};

// Thread 0, after qq = |q|^2: alpha and the scale of q.
__device__ __forceinline__ void cg_after_q(CgScalars& s, float qq) {
    int rs = 0;
    if (!isfinite(qq) || !(qq > 0.f)) {
        rs = kSegNonfinite;
    } else {
        s.alpha = s.rr / qq;
        vector_scale_f(qq, s.sc, s.inv);
    }
    s.reason = rs;
}

// Thread 0, after rr_new = |r|^2: segment end, or beta, pp and the scale of
// the next direction.
__device__ __forceinline__ void cg_after_r(CgScalars& s, float rr_new) {
    int rs = 0;
    s.it += 1;
    if (!isfinite(rr_new)) {
        rs = kSegNonfinite;
    } else if (rr_new <= s.stop || rr_new <= s.ru2 * s.rmax || s.it - s.it0 >= s.every) {
        rs = kSegUpdate;
    } else {
        const float b = rr_new / s.rr;
        s.beta = b;
        s.rr = rr_new;
        s.pp = fmaf(b * b, s.pp, rr_new);
        vector_scale_f(s.pp, s.sc, s.inv);
    }
    s.reason = rs;
}

// FP32 CG iterations of one segment (until a reliable update, max_iter or
// a non-finite norm) on split-K tiles with E' resident: M^dag contracts r
// (G = E r + beta G carried by the owners), M contracts u = e^{i phi} q.
// The owner vectors live in shared memory for the segment: r is loaded from
// the FP32 residual (or, refresh, the FP64 residual, also written back as
// FP32), p and G start at zero in the first segment of a solve and carry
// over otherwise, x (the FP32 increment) starts at zero and is folded into
// x64 by its owner at the end.
//
// Each application: wait for the owners of this CTA's K range (their posted
// words), copy and split the source with the scale from their largest
// exponent, issue the MMAs; meanwhile warp 0 sums the norm that the previous
// epilogue posted and thread 0 updates the scalars (alpha after |q|^2;
// beta, or the end of the segment, after |r|^2); then stage the partial,
// and, unless the segment ends, sync the cluster, reduce and run the
// epilogue, which writes the next source and posts its norm.  The decision
// to end the segment therefore comes after the next M^dag's MMAs are issued;
// their result is drained and dropped.  Returns the segment's end reason,
// or -1 if a bounded wait failed.  Not inlined into the persistent kernels:
// the iteration gets its own register budget.
__device__ __noinline__ int sk_segment(const ChainView& c, Team& ti, TcState& st,
                                       const PersistentArgs& pa, ClusterSync* ics,
                                       CgScalars& s_cg, bool refresh, bool first,
                                       const float2* cisf, double2* x64, float hop) {
    int reason = kSegMaxIter;
    const SkGeom g = sk_geom(ti.rank, pa.sk_C, pa.ns_tile, c.V, c.Nt, c.Vr, c.Vp);
    Team tcl = ti;
    tcl.rank = g.rank;
    tcl.size = g.C;
    tcl.cs = ics;
    SkOwner ow;
    ow.init(st.base, g);
    // the CTAs whose posts this CTA waits for: owners of the M^dag source (r)
    // and of the M source (u), and the other members of its cluster
    __shared__ int s_own[2][kSkMaxOwners];
    __shared__ int s_nown[2];
    __shared__ unsigned s_mexp;
    const CUtensorMap* maps = reinterpret_cast<const CUtensorMap*>(c.sk_maps);
    if (threadIdx.x == 0) {
        s_nown[0] = sk_owner_list(g, c.V, c.Nt, true, s_own[0], ti.rank);
        s_nown[1] = sk_owner_list(g, c.V, c.Nt, false, s_own[1], ti.rank);
        if (s_nown[0] < 0 || s_nown[1] < 0 || !maps) set_status(ti.status, HMC_ERR_UNSUPPORTED);
        if (maps)
            for (int m = 0; m < 6; ++m)
                asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(maps + m)
                             : "memory");
    }
    float2* rh = c.rh_f;   // r with the halo rows (source of M^dag)
    float mx = 0.f;
    HMC_SK_OWNED(o, oi, g, c) {
        float2 rv;
        if (refresh) {
            const double2 d = c.r[o];
            rv = make_float2((float)d.x, (float)d.y);
        } else {
            rv = c.r_f[o];
        }
        mx = fmaxf(mx, fmaxf(fabsf(rv.x), fabsf(rv.y)));
        const int t = (int)(o / (size_t)c.V);
        rh[o + c.V] = rv;                                        // row t + 1
        if (t == 0) rh[o + (size_t)(c.Nt + 1) * c.V] = rv;      // row Nt + 1
        ow.r[oi] = rv;
        ow.x[oi] = make_float2(0.f, 0.f);
        if (first) {
            ow.p[oi] = make_float2(0.f, 0.f);
            ow.G[oi] = make_float2(0.f, 0.f);
        }
    }
    sk_post(ti, c.gslots, ++st.gseq, 0.f, mx);   // r ready (no norm: beta is the caller's)
    if (team_failed(ti)) return -1;
    bool have_rr = false;
    const int warp = threadIdx.x >> 5;
    // Predicted operand exponents: s_pe[k] for the next source of kind k
    // (0: r, 1: u) from the team's largest exponent of its last one (every
    // CTA computes the same value from the same slots); s_pw[k]: the exponent
    // the owners used for the FP16 split of the last posted source of kind
    // k, or kNoPe if they wrote none (the segment's first r is FP32 only).
    constexpr int kNoPe = -1000;
    __shared__ int s_pe[2], s_pw[2];
    if (threadIdx.x == 0) {
        if (first) s_pe[0] = s_pe[1] = kNoPe;
        s_pw[0] = s_pw[1] = kNoPe;
    }
    // (the post above ended with a block barrier; these are read after the next)
    __half_raw* const b16 = c.sk_b16;
    const size_t plane = (size_t)2 * (c.Nt + 2) * c.Vp;
    // One application of kind `list` (0: M^dag, source r, halo rows t0 + 2 ..;
    // 1: M, source u, rows t0 ..): wait for the owners' words of seq; take
    // the owners' FP16 split by TMA when its exponent is known and the
    // owners' largest component scaled by it is in [2^4, 2^15) (no overflow,
    // full precision), else the FP32 source by TMA split here with the scale
    // from the owners' exponent; issue the MMAs.  Warp 1 sums the norm of seq
    // (into *out) and the team's largest exponent (into *gm) meanwhile.
    auto contract = [&](int list, float* out, unsigned* gm, float& inv) -> bool {
        if (warp == 0) {
            unsigned m = 0;
            const bool ok =
                sk_wait_owners(ti, c.gslots, st.gseq, s_own[list], s_nown[list], 0u, m);
            if ((threadIdx.x & 31) == 0) s_mexp = ok ? m : 0xffffffffu;
        }
        __syncthreads();
        const unsigned mexp = s_mexp;
        if (mexp == 0xffffffffu) return false;
        SkSum ss;
        if (warp == 1) sk_sum_begin(ti, c.gslots, st.gseq, ss);
        const int pw = s_pw[list];
        const int top = (int)mexp - 127 + pw;
        const bool fast = b16 && pw != kNoPe && mexp != 0xffu && (mexp == 0u || (top >= 4 && top <= 14));
        bool ok = true;
        const int row0 = list == 0 ? g.t0 + 2 : g.t0;
        if (fast) {
            inv = __int_as_float((127 - pw) << 23);
            sk_issue_b16(st, g, maps + 2 + 2 * list, maps + 3 + 2 * list, 2 * row0,
                         st.bars->tmem_base);
        } else {
            float sc;
            sk_scale(mexp, sc, inv);
            sk_issue_source(st, g, maps + list, row0);
            ok = sk_convert_and_issue(st, g, sc, st.bars->tmem_base);
        }
        if (ok && warp == 1) {
            float v = 0.f;
            unsigned gmx = 0;
            const bool oks = sk_sum_end(ti, c.gslots, st.gseq, ss, v, gmx);
            if ((threadIdx.x & 31) == 0) {
                *out = oks ? v : __int_as_float(0x7fc00000);
                *gm = gmx;
            }
        }
        return ok;
    };
    // predicted exponent of the next source of a kind whose largest
    // component had biased exponent gm: that component times 2^e in [2^12, 2^13)
    auto predict = [](unsigned gm) -> int {
        if (gm == 0u || gm == 0xffu) return kNoPe;
        return max(-120, min(120, 12 - ((int)gm - 127)));
    };
    __shared__ float s_norm;
    __shared__ unsigned s_gm;
    while (s_cg.it < pa.max_iter) {
        float inv;
        // ---- M^dag p' (p' = r + beta p): contract r
        if (!contract(0, &s_norm, &s_gm, inv)) return -1;
        __syncthreads();
        if (threadIdx.x == 0) {
            s_pe[0] = predict(s_gm);
            if (have_rr) {
                cg_after_r(s_cg, s_norm);
                if (s_cg.reason == 0 && s_cg.it >= pa.max_iter) s_cg.reason = kSegMaxIter;
            }
        }
        if (!sk_stage(st, g, inv)) return -1;   // its barrier publishes s_cg, s_pe
        if (team_failed(ti)) return -1;
        if (have_rr && s_cg.reason != 0) { reason = s_cg.reason; break; }
        const int pu = s_pe[1];
        SkEpiDag ed{ow, c.u_f, pu != kNoPe ? b16 + 2 * plane : nullptr, b16 + 3 * plane,
                    __int_as_float((127 + (pu != kNoPe ? pu : 0)) << 23), c.Vp,
                    cisf, s_cg.beta, hop, c.V, c.Nt, 0.f, 0.f};
        if (!sk_reduce<false>(st, g, tcl, c.V, c.e_inv, ed)) return -1;
        if (threadIdx.x == 0) s_pw[1] = b16 ? pu : kNoPe;
        sk_post(ti, c.gslots, ++st.gseq, ed.acc, ed.mx);   // u ready, |q|^2
        // ---- M q: contract u = e^{i phi} q
        if (!contract(1, &s_norm, &s_gm, inv)) return -1;
        __syncthreads();
        if (threadIdx.x == 0) {
            s_pe[1] = predict(s_gm);
            cg_after_q(s_cg, s_norm);
        }
        if (!sk_stage(st, g, inv)) return -1;
        if (team_failed(ti)) return -1;
        if (s_cg.reason != 0) { reason = s_cg.reason; break; }
        const int pr = s_pe[0];
        SkEpiM em{ow, rh, pr != kNoPe ? b16 : nullptr, b16 + plane,
                  __int_as_float((127 + (pr != kNoPe ? pr : 0)) << 23), c.Vp,
                  s_cg.alpha, hop, c.V, c.Nt, 0.f, 0.f};
        if (!sk_reduce<false>(st, g, tcl, c.V, c.e_inv, em)) return -1;
        if (threadIdx.x == 0) s_pw[0] = b16 ? pr : kNoPe;
        sk_post(ti, c.gslots, ++st.gseq, em.acc, em.mx);   // r ready, |r|^2
        have_rr = true;
    }
    if (reason != kSegNonfinite) {
        HMC_SK_OWNED(o, oi, g, c) {
            const float2 d = ow.x[oi];
            double2 xv = x64[o];
            xv.x += (double)d.x;
            xv.y += (double)d.y;
            x64[o] = xv;
        }
    }
    return reason;
}

// Kernel kinds of the FP32 iterations: site-major tensor-core tiles, the
// CUDA-core cluster solver, slice-major tensor-core tiles.
enum TileKind : int { kKindSite = 0, kKindSmall = 1, kKindSlice = 2, kKindSplitK = 3 };

template <int KIND>
__device__ bool cg_mixed(const ChainView& c, Team& tm, TcState& st, f64::Smem& sm64,
                         const CUtensorMap* mhi, const CUtensorMap* mlo,
                         const PersistentArgs& pa, ClusterSync* ics, const double2* chi,
                         double2* x64, MixedResult& res, bool warm = false, double gm1 = 0.0) {
    // the heavy operator M_g of mass preconditioning (gm1 = g - 1 != 0) is
    // built into the split-K tiles' epilogues only
    if (gm1 != 0.0 && KIND != kKindSplitK) {
        set_status(tm.status, HMC_ERR_UNSUPPORTED);
        return false;
    }
    constexpr bool SMALL = KIND == kKindSmall;
    float2 *rf = c.r_f, *pf = c.p_f, *pn = c.p2_f, *qf = c.q_f, *xf = c.x_f;
    const int inner_size = min(max(pa.inner, 1), tm.size);
    const bool in_inner = tm.rank < inner_size;
    Team ti = tm;
    ti.size = inner_size;
    ti.bar = c.bar + 2;
    // inner team = cluster 0: its barriers stay inside the cluster
    ti.cs = (ics && pa.cluster > 1 && inner_size == pa.cluster) ? ics : nullptr;
    // FP64 solution and |chi|^2 on all CTAs
    double v1[1] = {0.0};
    HMC_TEAM_ELEMS(e, c, tm) {
        const double2 ch = chi[e];
        if (!warm) x64[e] = make_double2(0.0, 0.0);
        v1[0] += ch.x * ch.x + ch.y * ch.y;
    }
    if (!team_sum<1>(tm, v1)) return false;
    const double chi2 = v1[0];
    res.iterations = 0;
    res.reliable_updates = 0;
    res.status = HMC_OK;
    res.true_res = 0.0;
    if (!(chi2 > 0.0)) {
        if (!finite_d(chi2)) res.status = HMC_ERR_NONFINITE;
        return true;
    }
    const double stop = pa.tol * pa.tol * chi2;
    // warm start (a later solve of a trajectory: same chi, the field moved by
    // one MD step): the FP64 true residual of the given x64 is the starting
    // residual of the FP32 iteration
    double rr_true = chi2;
    const double2* r0 = chi;
    if (warm) {
        if (!f64_residual(c, tm, sm64, chi, x64, rr_true, gm1)) return false;
        ++res.reliable_updates;
        if (!finite_d(rr_true)) {
            res.status = HMC_ERR_NONFINITE;
            return true;
        }
        if (rr_true <= stop) {
            res.true_res = sqrt(rr_true / chi2);
            return true;
        }
        r0 = c.r;
    }
    // FP32 iterates on the inner team (their owners).  A chain solved by one
    // CTA with E resident keeps them in shared memory: r, p, p', q, x and the
    // FP32 phase table, six vectors after the B ring.
    double rr = 0.0;
    const float2* cisf = c.cis_f;
    SmallCg sm;
    if constexpr (SMALL) {
      if (in_inner) {
        // small lattice: FP32 iterates of the cluster's slices in shared memory
        small_init_view(sm, st.base, tm.rank, inner_size, c.V, c.Nt);
        double v2[1] = {small_setup(sm, c, r0)};
        if (!team_sum<1>(ti, v2)) return false;
        rr = v2[0];
      }
    } else if (KIND == kKindSplitK && in_inner) {
        // split-K: this CTA's part of E' stays resident for the whole launch
        if (!st.sk_loaded) {
            const SkGeom g = sk_geom(tm.rank, pa.sk_C, pa.ns_tile, c.V, c.Nt, c.Vr, c.Vp);
            if (!sk_load_E(st, g, mhi, mlo)) return false;
            st.sk_loaded = 1;
        }
        double v2[1] = {0.0};
        HMC_TEAM_ELEMS(e, c, ti) {
            const double2 ch = r0[e];
            const float2 rv = make_float2((float)ch.x, (float)ch.y);
            rf[e] = rv;
            pf[e] = make_float2(0.f, 0.f);
            xf[e] = make_float2(0.f, 0.f);
            c.g_f[e] = make_float2(0.f, 0.f);
            v2[0] += (double)rv.x * rv.x + (double)rv.y * rv.y;
        }
        if (!team_sum<1>(ti, v2)) return false;
        rr = v2[0];
    } else if (in_inner) {
        if (pa.mode == kResident) {
            if (!tc_load_resident(st, mhi, mlo, (tm.rank % (c.Vr / TM)) * TM, c.Vp / KCH))
                return false;
        } else {
            tc_set_layout(st, kStreaming, 0);
        }
        if (pa.vec_resident) {
            float2* sv = reinterpret_cast<float2*>(st.free_area());
            rf = sv;
            pf = sv + c.N;
            pn = sv + 2 * c.N;
            qf = sv + 3 * c.N;
            xf = sv + 4 * c.N;
            float2* cs = sv + 5 * c.N;
            for (int e = threadIdx.x; e < c.N; e += blockDim.x) cs[e] = c.cis_f[e];
            cisf = cs;
        }
        double v2[1] = {0.0};
        HMC_TEAM_ELEMS(e, c, ti) {
            const double2 ch = r0[e];
            const float2 rv = make_float2((float)ch.x, (float)ch.y);
            rf[e] = rv;
            pf[e] = make_float2(0.f, 0.f);
            xf[e] = make_float2(0.f, 0.f);
            v2[0] += (double)rv.x * rv.x + (double)rv.y * rv.y;
        }
        if (!team_sum<1>(ti, v2)) return false;
        rr = v2[0];
    }
    __shared__ CgScalars s_cg;
    bool refresh = false;
    if (threadIdx.x == 0) {
        s_cg.rr = (float)rr;
        s_cg.pp = (float)rr;
        s_cg.rmax = (float)rr;
        s_cg.beta = 0.f;
        s_cg.stop = (float)stop;
        s_cg.ru2 = (float)(pa.ru_delta * pa.ru_delta);
        s_cg.it = 0;
        s_cg.it0 = 0;
        s_cg.every = pa.ru_every > 0 ? pa.ru_every : 1000;
        vector_scale(rr, s_cg.sc, s_cg.inv);
    }
    __syncthreads();
    bool conv = false;
    bool sk_first = true;   // split-K: the first segment starts p and G at zero
    // progress of the FP64 true residual between reliable updates: two
    // updates in a row that did not halve it mean the FP32 recursion has
    // stalled (near a singular M); the rest of the solve then runs in FP64
    double rr_last = rr_true;
    int stalls = 0;
    bool fallback = false;
    res.fp64_iterations = 0;
    volatile double* seg = c.scalars + 12;   // [0] end reason, [1] iterations
    for (;;) {
        if (SMALL && in_inner) {
            // small lattice: each half iteration is epilogue -> partial norm
            // out -> contraction -> boundary column out -> wait (byte-counted)
            __shared__ SmallSum s_ss;
            int reason = 0;
            if (refresh) {
                small_refresh_r(sm, c.r);
                refresh = false;
            }
            __syncthreads();
            small_load_ud(sm);
            __syncthreads();
            small_matvec_any(sm, sm.v(sm.l.ud));
            __syncthreads();
            small_send_boundary_plain(sm);
            if (!team_barrier(ti)) return false;   // boundary columns published
            unsigned kk = ti.cs ? ti.cs->count_tx : 0u;   // exchange phase
            const uint32_t xbytes = (uint32_t)(4 * ti.size + 8 * c.V);
            if (s_cg.it >= pa.max_iter) reason = kSegMaxIter;
            while (reason == 0) {
                float qq, rr_new;
                // q = M^dag p', p' = r + beta p; then E e^{i phi} q
                small_sum_begin(ti, s_ss, kk, small_dag_epilogue(sm, s_cg.beta));
                small_matvec_any(sm, sm.v(sm.l.um));
                __syncthreads();
                small_send_boundary(sm, ti.cs, kk, sm.S - 1, sm.l.bm, sm.next);
                if (!small_sum_end(ti, s_ss, kk, xbytes, qq)) return false;
                ++kk;
                if (threadIdx.x == 0) cg_after_q(s_cg, qq);
                __syncthreads();
                if (s_cg.reason != 0) { reason = s_cg.reason; break; }
                // x += alpha p', r -= alpha M q; then E r
                small_sum_begin(ti, s_ss, kk, small_m_epilogue(sm, s_cg.alpha));
                small_matvec_any(sm, sm.v(sm.l.ud));
                __syncthreads();
                small_send_boundary(sm, ti.cs, kk, 0, sm.l.bd, sm.prev);
                if (!small_sum_end(ti, s_ss, kk, xbytes, rr_new)) return false;
                ++kk;
                if (threadIdx.x == 0) {
                    cg_after_r(s_cg, rr_new);
                    if (s_cg.reason == 0 && s_cg.it >= pa.max_iter) s_cg.reason = kSegMaxIter;
                }
                __syncthreads();
                if (s_cg.reason != 0) { reason = s_cg.reason; break; }
            }
            if (threadIdx.x == 0 && ti.cs) ti.cs->count_tx = kk;
            if (reason != kSegNonfinite) small_fold_x(sm, x64);
            if (tm.rank == 0 && threadIdx.x == 0) {
                seg[0] = reason;
                seg[1] = s_cg.it;
            }
        } else if (KIND == kKindSplitK && in_inner) {
            const int reason = sk_segment(c, ti, st, pa, ics, s_cg, refresh, sk_first, cisf, x64,
                                          (float)(1.0 + gm1));
            if (reason < 0) return false;
            refresh = false;
            sk_first = false;
            if (tm.rank == 0 && threadIdx.x == 0) {
                seg[0] = reason;
                seg[1] = s_cg.it;
            }
        } else if (!SMALL && in_inner) {
            int reason = kSegMaxIter;
            while (s_cg.it < pa.max_iter) {
                // p_new = r + beta p; q = M^dag p_new
                SrcDirection dir{rf, c.r, pf, s_cg.beta, refresh, c.V};
                EpiDirection ed{dir, pn, rf, qf, cisf, c.Nt, 0.f};
                bool aok;
                if constexpr (KIND == kKindSlice)
                    aok = apply_team_w<true>(c, ti, st, pa.wide_W, mhi, mlo, pa.ns_tile, dir,
                                             s_cg.sc, s_cg.inv, ed);
                else
                    aok = apply_team<true>(c, ti, st, mhi, mlo, pa.ns_tile, dir, s_cg.sc,
                                           s_cg.inv, ed, pa.res_b != 0);
                if (!aok) return false;
                float qq;
                if (!team_sum_f(ti, ed.acc, qq)) return false;
                float2* t = pf;
                pf = pn;
                pn = t;
                refresh = false;
                if (threadIdx.x == 0) cg_after_q(s_cg, qq);
                __syncthreads();
                if (s_cg.reason != 0) { reason = s_cg.reason; break; }
                // Ap = M q; x += alpha p; r -= alpha Ap
                SrcPhase srcq{qf, cisf, c.V};
                EpiCgUpdate eu{qf, pf, xf, rf, s_cg.alpha, c.V, 0.f};
                if constexpr (KIND == kKindSlice)
                    aok = apply_team_w<false>(c, ti, st, pa.wide_W, mhi, mlo, pa.ns_tile, srcq,
                                              s_cg.sc, s_cg.inv, eu);
                else
                    aok = apply_team<false>(c, ti, st, mhi, mlo, pa.ns_tile, srcq, s_cg.sc,
                                            s_cg.inv, eu, pa.res_b != 0);
                if (!aok) return false;
                float rr_new;
                if (!team_sum_f(ti, eu.acc, rr_new)) return false;
                if (threadIdx.x == 0) cg_after_r(s_cg, rr_new);
                __syncthreads();
                if (s_cg.reason != 0) { reason = s_cg.reason; break; }
            }
            // fold the FP32 increment into x64 (the inner team owns x_f)
            if (reason != kSegNonfinite) {
                HMC_TEAM_ELEMS(e, c, ti) {
                    const float2 d = xf[e];
                    double2 xv = x64[e];
                    xv.x += (double)d.x;
                    xv.y += (double)d.y;
                    x64[e] = xv;
                    xf[e] = make_float2(0.f, 0.f);
                }
            }
            if (tm.rank == 0 && threadIdx.x == 0) {
                seg[0] = reason;
                seg[1] = s_cg.it;
            }
        }
        if (!team_barrier(tm)) return false;
        const int reason = (int)seg[0];
        const int it = (int)seg[1];
        if (reason == kSegNonfinite) { res.status = HMC_ERR_NONFINITE; break; }
        // FP64 true residual on all CTAs
        if (!f64_residual(c, tm, sm64, chi, x64, rr_true, gm1)) return false;
        ++res.reliable_updates;
        if (!finite_d(rr_true)) { res.status = HMC_ERR_NONFINITE; break; }
        if (rr_true <= stop) { conv = true; break; }
        if (reason == kSegMaxIter) break;
        stalls = rr_true > 0.25 * rr_last ? stalls + 1 : 0;
        rr_last = rr_true;
        if (stalls >= 2) { fallback = true; break; }
        // continue from the true residual; keep the direction
        if (threadIdx.x == 0) {
            const double b = rr_true / (double)s_cg.rr;
            const double pp = rr_true + b * b * (double)s_cg.pp;
            s_cg.beta = (float)b;
            s_cg.rr = (float)rr_true;
            s_cg.rmax = (float)rr_true;
            s_cg.pp = (float)pp;
            s_cg.it = it;
            s_cg.it0 = it;
            vector_scale(pp, s_cg.sc, s_cg.inv);
        }
        __syncthreads();
        refresh = true;
    }
    res.iterations = (int)seg[1];
    if (fallback) {
        // FP64 CG on all CTAs from the current solution; its final true
        // residual leaves M^dag x in q, as the reliable update does
        f64::CgResult r64;
        if (!f64::cg_solve(c, tm, chi, x64, pa.tol, max(1, pa.max_iter - res.iterations), r64,
                           sm64, true, gm1))
            return false;
        res.fp64_iterations = r64.iterations;
        res.true_res = r64.true_res;
        res.status = r64.status;
        return true;
    }
    if (!conv && res.status == HMC_OK) res.status = HMC_ERR_CG_NOT_CONVERGED;
    res.true_res = sqrt(rr_true / chi2);
    if (!finite_d(res.true_res)) res.status = HMC_ERR_NONFINITE;
    return true;
}

// Cluster launch: set up the cluster team state and check that the inner
// team's ranks are the cluster ranks of cluster 0.
__device__ inline void cluster_begin(const PersistentArgs& pa, ClusterSync* cs, int* status) {
    if (pa.cluster <= 1) return;
    if (threadIdx.x == 0 && cluster_ctarank() != (uint32_t)(blockIdx.x % pa.cluster))
        set_status(status, HMC_ERR_UNSUPPORTED);
    cluster_sync_init(cs, pa.cluster);
}

__device__ __forceinline__ Team make_team(const ChainView& c) {
    Team tm;
    tm.rank = blockIdx.x;
    tm.size = gridDim.x + c.team_pad;
    tm.bar = c.bar;
    tm.status = c.status;
    tm.partials = c.partials;
    tm.cs = nullptr;
    return tm;
}

__device__ __forceinline__ void set_phases(const ChainView& c, const Team& tm,
                                           const double* phi) {
    HMC_TEAM_ELEMS(e, c, tm) {
        double s, co;
        sincos(phi[e], &s, &co);
        c.cis[e] = make_double2(co, s);
        c.cis_f[e] = make_float2((float)co, (float)s);
    }
}

// Per-launch set-up of the operand area: the tensor-core path takes its
// mbarriers and TMEM; the small (CUDA-core) mode needs only the area.
template <bool SMALL>
__device__ inline void persistent_setup(TcState& st, uint8_t* dyn, int* status) {
    if constexpr (SMALL) {
        st.base = smem_base(dyn);
        st.status = status;
        st.ntile = 0;
    } else {
        tc_setup(st, dyn, status);
    }
}
template <bool SMALL>
__device__ inline void persistent_teardown(TcState& st) {
    if constexpr (!SMALL) tc_teardown(st);
}

// scalars: [0] iterations [1] true residual [2] status [3] reliable updates
// KIND: TileKind of the FP32 iterations.
template <int KIND>
__global__ void __launch_bounds__(NTHR, 1)
    k_cg(const __grid_constant__ CUtensorMap mhi, const __grid_constant__ CUtensorMap mlo,
         ChainView c, PersistentArgs pa, const double* phi, const double2* chi, double2* x) {
    extern __shared__ __align__(1024) uint8_t dyn[];
    __shared__ f64::Smem sm64;
    TcState st;
    persistent_setup<KIND == kKindSmall>(st, dyn, c.status);
    __shared__ ClusterSync s_cs;
    Team tm = make_team(c);
    cluster_begin(pa, &s_cs, c.status);
    set_phases(c, tm, phi);
    MixedResult res{};
    bool ok = team_barrier(tm);
    if (ok) ok = cg_mixed<KIND>(c, tm, st, sm64, &mhi, &mlo, pa, &s_cs, chi, x, res);
    if (ok && tm.rank == 0 && threadIdx.x == 0) {
        c.scalars[0] = res.iterations;
        c.scalars[1] = res.true_res;
        c.scalars[2] = res.status;
        c.scalars[3] = res.reliable_updates;
        c.scalars[4] = res.fp64_iterations;
    }
    persistent_teardown<KIND == kKindSmall>(st);
    if (pa.cluster > 1) cluster_barrier_all();   // no member leaves while others may push
}

// One HMC trajectory with the mixed solver (same steps as the FP64 one),
// run by team `tm`; results in c.scalars.  Returns false if the team failed.
template <int KIND>
__device__ bool run_trajectory(const ChainView& c, Team& tm, TcState& st, f64::Smem& sm64,
                               const CUtensorMap* mhi, const CUtensorMap* mlo,
                               const PersistentArgs& pa, ClusterSync* ics, const TrajArgs& a) {
    double* phi = a.phi;
    const double inv_dU = 1.0 / (c.delta * c.U);
    const double rsqrt2 = 0.70710678118654752440;
    double h0[3] = {0.0, 0.0, 0.0};
    HMC_TEAM_ELEMS(e, c, tm) {
        const double2 zp = normal_pair(philox_draw(a.seed, kStreamMomentum, a.traj, a.chain, e));
        const double2 zr = normal_pair(philox_draw(a.seed, kStreamNoise, a.traj, a.chain, e));
        const double ph = phi[e];
        c.pi[e] = zp.x;
        const double2 rho = make_double2(zr.x * rsqrt2, zr.y * rsqrt2);
        c.rho[e] = rho;
        c.phi_old[e] = ph;
        double s, co;
        sincos(ph, &s, &co);
        c.cis[e] = make_double2(co, s);
        c.cis_f[e] = make_float2((float)co, (float)s);
        h0[0] += ph * ph;
        h0[1] += rho.x * rho.x + rho.y * rho.y;
        h0[2] += zp.x * zp.x;
    }
    bool ok = team_sum<3>(tm, h0);
    const double H0 = 0.5 * h0[0] * inv_dU + h0[1] + 0.5 * h0[2];
    f64::EpiArgs ea = {};
    if (ok) {
        f64::apply_team<false, f64::EPI_STORE>(c, tm, c.rho, c.chi, ea, sm64);
        ok = team_barrier(tm);
    }
    int iters = 0, solves = 0, rus = 0, fp64_iters = 0, status = HMC_OK;
    double max_res = 0.0;
    ea.phi = phi;
    ea.pi = c.pi;
    ea.inv_dU = inv_dU;
    const double ed = a.eps * c.delta;
    const double edrift = md_drift(a) * ed;
    const int n_stages = md_stages(a);
    // initial guesses of the solves (the solves sit at equally spaced fields):
    // the first from zero, the second from the first solution, the third
    // from the linear extrapolation 2 x_{k-1} - x_{k-2}, later ones from the
    // quadratic one 3 x_{k-1} - 3 x_{k-2} + x_{k-3}; rho, free once chi and
    // H0 are formed, keeps x_{k-2}, xh keeps x_{k-3}
    double2* xold = c.rho;
    for (int step = 0; ok && step <= n_stages; ++step) {
        if (step > 0) {
            HMC_TEAM_ELEMS(e, c, tm) {
                const double ph = fma(edrift, c.pi[e], phi[e]);
                phi[e] = ph;
                double s, co;
                sincos(ph, &s, &co);
                c.cis[e] = make_double2(co, s);
                c.cis_f[e] = make_float2((float)co, (float)s);
                const double2 x1 = c.x[e];
                if (step > 2) {
                    const double2 x2 = xold[e], x3 = c.xh[e];
                    c.x[e] = make_double2(3.0 * (x1.x - x2.x) + x3.x, 3.0 * (x1.y - x2.y) + x3.y);
                    c.xh[e] = x2;
                } else if (step > 1) {
                    const double2 x2 = xold[e];
                    c.x[e] = make_double2(2.0 * x1.x - x2.x, 2.0 * x1.y - x2.y);
                    c.xh[e] = x2;
                }
                xold[e] = x1;
            }
            if (!(ok = team_barrier(tm))) break;
        }
        MixedResult res{};
        if (!(ok = cg_mixed<KIND>(c, tm, st, sm64, mhi, mlo, pa, ics, c.chi, c.x, res, step > 0)))
            break;
        iters += res.iterations;
        rus += res.reliable_updates;
        fp64_iters += res.fp64_iterations;
        ++solves;
        max_res = fmax(max_res, res.true_res);
        if (res.status != HMC_OK && status == HMC_OK) status = res.status;
        ea.kick = md_kick(a, step) * ed;
        if (res.status == HMC_OK) {
            // the solve ended on an FP64 true residual of its final x, which
            // left q = M^dag x (same FP64 tile): the force needs no
            // application of its own
            HMC_TEAM_ELEMS(e, c, tm) {
                const double2 xv = c.x[e], y = c.q[e];
                const double f = phi[e] * inv_dU + 2.0 * (xv.y * y.x - xv.x * y.y);
                c.pi[e] -= ea.kick * f;
            }
        } else {
            f64::apply_team<true, f64::EPI_FORCE>(c, tm, c.x, nullptr, ea, sm64);
        }
        ok = team_barrier(tm);
    }
    double h1[3] = {0.0, 0.0, 0.0};
    if (ok) {
        HMC_TEAM_ELEMS(e, c, tm) {
            const double ph = phi[e], pv = c.pi[e];
            const double2 ch = c.chi[e], xv = c.x[e];
            h1[0] += ph * ph;
            h1[1] += ch.x * xv.x + ch.y * xv.y;
            h1[2] += pv * pv;
        }
        ok = team_sum<3>(tm, h1);
    }
    if (ok) {
        const double H1 = 0.5 * h1[0] * inv_dU + h1[1] + 0.5 * h1[2];
        const double dH = H1 - H0;
        const double u =
            uniform_pair(philox_draw(a.seed, kStreamMetropolis, a.traj, a.chain, 0)).x;
        const bool accept = u < exp(-dH);
        if (!accept) {
            HMC_TEAM_ELEMS(e, c, tm) phi[e] = c.phi_old[e];
        }
        if (tm.rank == 0 && threadIdx.x == 0) {
            c.scalars[kTrajDH] = dH;
            c.scalars[kTrajH0] = H0;
            c.scalars[kTrajH1] = H1;
            c.scalars[kTrajU] = u;
            c.scalars[kTrajAccept] = accept ? 1.0 : 0.0;
            c.scalars[kTrajIters] = iters;
            c.scalars[kTrajSolves] = solves;
            c.scalars[kTrajRU] = rus;
            c.scalars[kTrajMaxRes] = max_res;
            c.scalars[kTrajStatus] = status;
            c.scalars[kTrajFp64Iters] = fp64_iters;
        }
    }
    return ok;
}

// One HMC trajectory with mass preconditioning (Hasenbusch 2001) and the
// two-level nested leapfrog (Sexton and Weingarten 1992) on the mixed path:
// the same steps as f64::k_trajectory_hb, with every solve the mixed CG
// (FP32 iterations on the split-K tiles, whose epilogues scale the
// contraction by g for the heavy operator M_g = 1 - g S E D; FP64 reliable
// updates and true residuals of the same operator) and everything else in
// FP64.  Each solve's final FP64 residual leaves q = (M_g or M)^dag x, from
// which the forces are formed.  The first solve of each level starts from
// zero, the later ones from that level's previous solution (same right-hand
// side on the inner level; consecutive solves of a level sit one step of
// that level apart).  Results in c.scalars as the FP64 kernel's.
template <int KIND>
__device__ __noinline__ bool run_trajectory_hb(const ChainView& c, Team& tm, TcState& st,
                                              f64::Smem& sm64,
                                  const CUtensorMap* mhi, const CUtensorMap* mlo,
                                  const PersistentArgs& pa, ClusterSync* ics,
                                  const TrajArgs& a) {
    double* phi = a.phi;
    const double inv_dU = 1.0 / (c.delta * c.U);
    const double rsqrt2 = 0.70710678118654752440;
    const double gm1 = a.hb_gamma - 1.0;
    // 1. heat bath: momenta, the two noise vectors (rho_1 from stream 3 in
    // c.rho, rho_2 from the plain noise stream in c.xh), start energy
    double h0[3] = {0.0, 0.0, 0.0};
    HMC_TEAM_ELEMS(e, c, tm) {
        const double2 zp = normal_pair(philox_draw(a.seed, kStreamMomentum, a.traj, a.chain, e));
        const double2 z2 = normal_pair(philox_draw(a.seed, kStreamNoise, a.traj, a.chain, e));
        const double2 z1 = normal_pair(philox_draw(a.seed, kStreamHeavy, a.traj, a.chain, e));
        const double ph = phi[e];
        c.pi[e] = zp.x;
        const double2 r1 = make_double2(z1.x * rsqrt2, z1.y * rsqrt2);
        const double2 r2 = make_double2(z2.x * rsqrt2, z2.y * rsqrt2);
        c.rho[e] = r1;
        c.xh[e] = r2;
        c.phi_old[e] = ph;
        double s, co;
        sincos(ph, &s, &co);
        c.cis[e] = make_double2(co, s);
        c.cis_f[e] = make_float2((float)co, (float)s);
        h0[0] += ph * ph;
        h0[1] += r1.x * r1.x + r1.y * r1.y + r2.x * r2.x + r2.y * r2.y;
        h0[2] += zp.x * zp.x;
    }
    if (!team_sum<3>(tm, h0)) return false;
    const double H0 = 0.5 * h0[0] * inv_dU + h0[1] + 0.5 * h0[2];
    int iters_in = 0, iters_out = 0, solves_in = 0, solves_out = 0, rus = 0, fp64_iters = 0;
    int status = HMC_OK;
    double max_res = 0.0;
    auto record = [&](const MixedResult& r, bool outer) {
        (outer ? iters_out : iters_in) += r.iterations;
        ++(outer ? solves_out : solves_in);
        rus += r.reliable_updates;
        fp64_iters += r.fp64_iterations;
        max_res = fmax(max_res, r.true_res);
        if (r.status != HMC_OK && status == HMC_OK) status = r.status;
    };
    // 2. chi_1 = M_g rho_1; chi_2 = M_g^dag (M_g M_g^dag)^{-1} M rho_2
    f64::EpiArgs eg = {};
    eg.hop_m1 = gm1;
    f64::EpiArgs e1 = {};
    f64::apply_team<false, f64::EPI_STORE>(c, tm, c.rho, c.chi, eg, sm64);
    f64::apply_team<false, f64::EPI_STORE>(c, tm, c.xh, c.phi2, e1, sm64);
    if (!team_barrier(tm)) return false;
    MixedResult res{};
    if (!cg_mixed<KIND>(c, tm, st, sm64, mhi, mlo, pa, ics, c.phi2, c.x2, res, false, gm1))
        return false;
    record(res, false);
    if (res.status == HMC_OK) {
        HMC_TEAM_ELEMS(e, c, tm) c.chi2[e] = c.q[e];   // q = M_g^dag x_2 (final residual)
    } else {
        f64::apply_team<true, f64::EPI_STORE>(c, tm, c.x2, c.chi2, eg, sm64);
    }
    if (!team_barrier(tm)) return false;
    // 3. nested leapfrog
    const double ed = a.eps * c.delta;
    const double h = 1.0 / a.hb_inner;
    auto drift = [&](double cf) {
        HMC_TEAM_ELEMS(e, c, tm) {
            const double ph = fma(cf * ed, c.pi[e], phi[e]);
            phi[e] = ph;
            double s, co;
            sincos(ph, &s, &co);
            c.cis[e] = make_double2(co, s);
            c.cis_f[e] = make_float2((float)co, (float)s);
        }
        return team_barrier(tm);
    };
    // bosonic and heavy forces: F_B + F_1 = phi/(delta U) + 2 Im(x_1 conj(M_g^dag x_1))
    bool warm_in = false, warm_out = false;
    auto kick_inner = [&](double cf) {
        MixedResult r{};
        if (!cg_mixed<KIND>(c, tm, st, sm64, mhi, mlo, pa, ics, c.chi, c.x, r, warm_in, gm1))
            return false;
        warm_in = true;
        record(r, false);
        const double k = cf * ed;
        if (r.status == HMC_OK) {
            HMC_TEAM_ELEMS(e, c, tm) {
                const double2 xv = c.x[e], y = c.q[e];
                c.pi[e] -= k * (phi[e] * inv_dU + 2.0 * (xv.y * y.x - xv.x * y.y));
            }
        } else {
            f64::EpiArgs ef = {};
            ef.hop_m1 = gm1;
            ef.phi = phi;
            ef.pi = c.pi;
            ef.inv_dU = inv_dU;
            ef.kick = k;
            f64::apply_team<true, f64::EPI_FORCE>(c, tm, c.x, nullptr, ef, sm64);
        }
        return team_barrier(tm);
    };
    // ratio force: F_2 = 2 Im(x_2 conj(M^dag x_2)) - 2 Im(conj(M_g^dag x_2 - x_2) chi_2)
    auto kick_outer = [&](double cf) {
        f64::apply_team<false, f64::EPI_STORE>(c, tm, c.chi2, c.phi2, eg, sm64);   // M_g chi_2
        if (!team_barrier(tm)) return false;
        MixedResult r{};
        if (!cg_mixed<KIND>(c, tm, st, sm64, mhi, mlo, pa, ics, c.phi2, c.x2, r, warm_out, 0.0))
            return false;
        warm_out = true;
        record(r, true);
        const double k = cf * ed;
        f64::EpiArgs ef = {};
        ef.phi = phi;
        ef.pi = c.pi;
        ef.inv_dU = 0.0;          // the bosonic force sits on the inner level
        ef.kick = k;
        if (r.status == HMC_OK) {
            HMC_TEAM_ELEMS(e, c, tm) {
                const double2 xv = c.x2[e], y = c.q[e];
                c.pi[e] -= k * (2.0 * (xv.y * y.x - xv.x * y.y));
            }
        } else {
            f64::apply_team<true, f64::EPI_FORCE>(c, tm, c.x2, nullptr, ef, sm64);
        }
        if (!team_barrier(tm)) return false;
        ef.hop_m1 = gm1;
        ef.chi = c.chi2;
        f64::apply_team<true, f64::EPI_RATIO>(c, tm, c.x2, nullptr, ef, sm64);
        return team_barrier(tm);
    };
    if (!kick_outer(0.5)) return false;
    for (int k = 0; k < a.n_md; ++k) {
        for (int m = 0; m < a.hb_inner; ++m) {
            if (!kick_inner(m == 0 ? 0.5 * h : h)) return false;
            if (!drift(h)) return false;
        }
        if (!kick_inner(0.5 * h)) return false;
        if (!kick_outer(k + 1 < a.n_md ? 1.0 : 0.5)) return false;
    }
    // 4. end energy (the last kick of each level was at the final field) and
    // Metropolis
    double h1[4] = {0.0, 0.0, 0.0, 0.0};
    HMC_TEAM_ELEMS(e, c, tm) {
        const double ph = phi[e], pv = c.pi[e];
        const double2 c1 = c.chi[e], x1 = c.x[e], p2 = c.phi2[e], x2 = c.x2[e];
        h1[0] += ph * ph;
        h1[1] += c1.x * x1.x + c1.y * x1.y;
        h1[2] += p2.x * x2.x + p2.y * x2.y;
        h1[3] += pv * pv;
    }
    if (!team_sum<4>(tm, h1)) return false;
    const double H1 = 0.5 * h1[0] * inv_dU + h1[1] + h1[2] + 0.5 * h1[3];
    const double dH = H1 - H0;
    const double u = uniform_pair(philox_draw(a.seed, kStreamMetropolis, a.traj, a.chain, 0)).x;
    const bool accept = u < exp(-dH);
    if (!accept) {
        HMC_TEAM_ELEMS(e, c, tm) phi[e] = c.phi_old[e];
    }
    if (tm.rank == 0 && threadIdx.x == 0) {
        c.scalars[kTrajDH] = dH;
        c.scalars[kTrajH0] = H0;
        c.scalars[kTrajH1] = H1;
        c.scalars[kTrajU] = u;
        c.scalars[kTrajAccept] = accept ? 1.0 : 0.0;
        c.scalars[kTrajIters] = iters_in + iters_out;
        c.scalars[kTrajSolves] = solves_in + solves_out;
        c.scalars[kTrajRU] = rus;
        c.scalars[kTrajMaxRes] = max_res;
        c.scalars[kTrajStatus] = status;
        c.scalars[kTrajFp64Iters] = fp64_iters;
        c.scalars[kTrajItersOuter] = iters_out;
        c.scalars[kTrajSolvesOuter] = solves_out;
    }
    return true;
}

template <int KIND>
__global__ void __launch_bounds__(NTHR, 1)
    k_trajectory(const __grid_constant__ CUtensorMap mhi,
                 const __grid_constant__ CUtensorMap mlo, ChainView c, PersistentArgs pa,
                 TrajArgs a) {
    extern __shared__ __align__(1024) uint8_t dyn[];
    __shared__ f64::Smem sm64;
    TcState st;
    persistent_setup<KIND == kKindSmall>(st, dyn, c.status);
    __shared__ ClusterSync s_cs;
    Team tm = make_team(c);
    cluster_begin(pa, &s_cs, c.status);
    if constexpr (KIND == kKindSplitK) {
        // (mass preconditioning: split-K tiles only; the host refuses it for
        // the other kinds)
        if (a.hb_inner > 0)
            run_trajectory_hb<KIND>(c, tm, st, sm64, &mhi, &mlo, pa, &s_cs, a);
        else
            run_trajectory<KIND>(c, tm, st, sm64, &mhi, &mlo, pa, &s_cs, a);
    } else {
        run_trajectory<KIND>(c, tm, st, sm64, &mhi, &mlo, pa, &s_cs, a);
    }
    persistent_teardown<KIND == kKindSmall>(st);
    if (pa.cluster > 1) cluster_barrier_all();   // no member leaves while others may push
}

// ---------------------------------------------------------------- batched
// Many independent chains of different sizes in one persistent launch,
// chains ordered by decreasing estimated cost.  With csize == 1 every CTA
// takes the next chain from an atomic work queue and runs its whole
// trajectory as a one-CTA team.  With csize > 1 the launch is made of
// thread-block clusters of csize CTAs and the queue starts with the chains
// marked as cluster teams (the most expensive ones): while those last, rank
// 0 of a cluster takes the next chain and hands its index to every member,
// and the cluster runs it as one team (barriers and sums through
// distributed shared memory, FP64 steps over all csize CTAs).  At the first
// one-CTA chain the cluster's members go their own way: rank 0 runs that
// chain and every member takes further chains alone.  The TMEM allocation
// and the operand ring persist across chains.
// One trajectory of a batch chain of kind KIND; not inlined, so each kind
// is compiled (and given registers) once, whichever phase runs it.
template <int KIND>
__device__ __noinline__ bool batch_traj(const BatchItem& it, TcState& st, f64::Smem& sm64,
                                        Team& tm, ClusterSync* ics, const TrajArgs& a) {
    const CUtensorMap* m = KIND == kKindSlice ? it.maps + 2 : it.maps;
    return run_trajectory<KIND>(it.v, tm, st, sm64, m, m + 1, it.pa, ics, a);
}

__device__ inline void batch_run(const BatchItem& it, int ci, const BatchCallArgs* call,
                                 double* outs, TcState& st, f64::Smem& sm64, Team& tm,
                                 ClusterSync* ics, bool write_out, bool& ok) {
    st.status = it.v.status;
    TrajArgs a = it.a;
    a.seed = call->seed;
    a.traj = call->traj;
    a.phi = call->phi + it.offset;
    if (it.pa.mode == kSmall)
        ok = batch_traj<kKindSmall>(it, st, sm64, tm, ics, a);
    else if (it.pa.mode == kSlice)
        ok = batch_traj<kKindSlice>(it, st, sm64, tm, ics, a);
    else
        ok = batch_traj<kKindSite>(it, st, sm64, tm, ics, a);
    __syncthreads();
    if (write_out && threadIdx.x == 0) {
        for (int k = 0; k < kNumScalars; ++k)
            outs[(size_t)ci * kNumScalars + k] = it.v.scalars[k];
        outs[(size_t)ci * kNumScalars + kTrajStatus] =
            ok ? it.v.scalars[kTrajStatus] : (double)(*((volatile int*)it.v.status));
    }
}

// Reset a chain's status and scalars and make its tensor maps (global
// memory) visible to the TMA proxy of this CTA.  Thread 0.
__device__ inline void batch_chain_begin(const BatchItem& it, bool reset) {
    if (reset) {
        *it.v.status = 0;
        for (int k = 0; k < kNumScalars; ++k) it.v.scalars[k] = 0.0;
    }
    for (int m = 0; m < 4; ++m)
        asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(it.maps + m)
                     : "memory");
}

__global__ void __launch_bounds__(NTHR, 1)
    k_batch(const BatchItem* __restrict__ items, const int* __restrict__ order, int n,
            int* queue, const BatchCallArgs* call, double* outs, int csize) {
    extern __shared__ __align__(1024) uint8_t dyn[];
    __shared__ f64::Smem sm64;
    __shared__ int s_idx;
    __shared__ ClusterSync s_cs;
    TcState st;
    tc_setup(st, dyn, items[0].v.status);
    const int crank = csize > 1 ? (int)cluster_ctarank() : 0;
    if (csize > 1) cluster_sync_init(&s_cs, csize);
    bool solo = csize == 1;
    bool ok = true;
    // cluster phase: one team chain per cluster at a time
    while (!solo) {
        if (crank == 0 && threadIdx.x == 0) {
            const int v = atomicAdd(queue, 1);
            if (v < n && items[order[v]].team > 1) batch_chain_begin(items[order[v]], true);
            const uint32_t la = cta_smem_u32(&s_idx);
            for (int r = 0; r < csize; ++r) {
                uint32_t ra;
                asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(la), "r"(r));
                asm volatile("st.shared::cluster.s32 [%0], %1;" ::"r"(ra), "r"(v) : "memory");
            }
        }
        cluster_barrier_all();          // the index (and the chain's reset) published
        const int idx = s_idx;
        cluster_barrier_all();          // read by every member before the next write
        if (idx >= n) break;
        const int ci = order[idx];
        const BatchItem& it = items[ci];
        if (it.team <= 1) {
            // first one-CTA chain: rank 0 runs it, then all members go alone
            solo = true;
            if (crank == 0) {
                if (threadIdx.x == 0) batch_chain_begin(it, true);
                __syncthreads();
                Team tm{};
                tm.rank = 0;
                tm.size = 1;
                tm.bar = it.v.bar;
                tm.status = it.v.status;
                tm.partials = it.v.partials;
                tm.cs = nullptr;
                batch_run(it, ci, call, outs, st, sm64, tm, nullptr, true, ok);
            }
            break;
        }
        if (threadIdx.x == 0 && crank != 0) batch_chain_begin(it, false);
        __syncthreads();
        Team tm{};
        tm.rank = crank;
        tm.size = csize;
        tm.bar = it.v.bar;
        tm.status = it.v.status;
        tm.partials = it.v.partials;
        tm.cs = &s_cs;
        batch_run(it, ci, call, outs, st, sm64, tm, &s_cs, crank == 0, ok);
        // the team's outcome, the same on every member: a failed member has
        // set the chain's status before it left its waits
        cluster_barrier_all();
        ok = *((volatile int*)it.v.status) == 0;
        if (!ok) break;
    }
    // one-CTA phase
    while (ok) {
        if (threadIdx.x == 0) s_idx = atomicAdd(queue, 1);
        __syncthreads();
        const int idx = s_idx;
        __syncthreads();
        if (idx >= n) break;
        const int ci = order[idx];
        const BatchItem& it = items[ci];
        if (threadIdx.x == 0) batch_chain_begin(it, true);
        __syncthreads();
        Team tm{};
        tm.rank = 0;
        tm.size = 1;
        tm.bar = it.v.bar;
        tm.status = it.v.status;
        tm.partials = it.v.partials;
        tm.cs = nullptr;
        batch_run(it, ci, call, outs, st, sm64, tm, nullptr, true, ok);
        // a failed bounded wait leaves the operand ring in an unknown phase:
        // this CTA takes no further chains (they stay unprocessed, status set)
    }
    tc_teardown(st);
    if (csize > 1) cluster_barrier_all();   // no member leaves while others may push to it
}
}  // namespace tc

// ---------------------------------------------------------------- host side
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    }
    return fn;
}

static bool splitk_shape(const hmc_ctx* c, int* C_out, int* ns_out);

static bool make_map(CUtensorMap* m, void* base, int Vr, int Vp, int box_rows = tc::TM) {
    auto enc = encode_fn();
    if (!enc) return false;
    cuuint64_t dims[2] = {(cuuint64_t)Vp, (cuuint64_t)Vr};
    cuuint64_t strides[1] = {(cuuint64_t)Vp * 2};
    cuuint32_t box[2] = {(cuuint32_t)tc::KCH, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, base, dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
           CUDA_SUCCESS;
}

// TMA map of a split-K source with halo rows: [rows][V] complex64 seen as
// 8-byte integers (the bits are copied as they are), boxes of 64 sites x
// box_rows rows, no swizzle, zero fill outside.
static bool make_map_src(CUtensorMap* m, void* base, int rows, int V, int box_rows) {
    auto enc = encode_fn();
    if (!enc) return false;
    cuuint64_t dims[2] = {(cuuint64_t)V, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)V * 8};
    cuuint32_t box[2] = {(cuuint32_t)tc::KCH, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_INT64, 2, base, dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
               CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
           CUDA_SUCCESS;
}

// Smallest slices-per-tile in {8, 16, 32, 64} with at most `slots` tiles.
static int pick_ns(int nti, int Nt, int slots) {
    int ns = 8;
    while (ns < tc::NMAX / 2 && nti * ((Nt + ns - 1) / ns) > slots) ns *= 2;
    return ns;
}

static void* dev_alloc(hmc_ctx* c, size_t bytes, bool* ok) {
    if (!*ok) return nullptr;
    void* p = nullptr;
    if (c->n_allocs >= (int)(sizeof(c->allocs) / sizeof(c->allocs[0])) ||
        cudaMalloc(&p, bytes) != cudaSuccess) {
        *ok = false;
        return nullptr;
    }
    c->allocs[c->n_allocs++] = p;
    cudaMemset(p, 0, bytes);
    return p;
}

int tc_ctx_init(hmc_ctx* c) {
    ChainView& v = c->view;
    const int V = v.V;
    v.Vr = ((V + tc::TM - 1) / tc::TM) * tc::TM;
    v.Vp = ((V + tc::KCH - 1) / tc::KCH) * tc::KCH;
    std::vector<double> E((size_t)V * V);
    if (cudaMemcpy(E.data(), v.E, E.size() * sizeof(double), cudaMemcpyDeviceToHost) !=
        cudaSuccess)
        return HMC_ERR_CUDA;
    // E = E_hi + 2^-11 E_lo with both parts in fp16, padded with zeros
    std::vector<__half> hi((size_t)v.Vr * v.Vp), lo((size_t)v.Vr * v.Vp);
    for (int r = 0; r < v.Vr; ++r)
        for (int k = 0; k < v.Vp; ++k) {
            const double e = (r < V && k < V) ? E[(size_t)r * V + k] : 0.0;
            const __half h = __float2half_rn((float)e);
            const double rem = (e - (double)__half2float(h)) * 2048.0;
            hi[(size_t)r * v.Vp + k] = h;
            lo[(size_t)r * v.Vp + k] = __float2half_rn((float)rem);
        }
    // slice-major tile: 2^eE E = Ew_hi + Ew_lo (plain remainder) with
    // max |2^eE E| in [2^14, 2^15)
    double emax = 0.0;
    for (size_t k = 0; k < E.size(); ++k) emax = std::max(emax, std::fabs(E[k]));
    int eE = 0;
    if (emax > 0.0 && std::isfinite(emax)) {
        int ex = 0;
        std::frexp(emax, &ex);   // emax in [2^(ex-1), 2^ex)
        eE = std::max(-100, std::min(100, 15 - ex));
    }
    const double es = std::ldexp(1.0, eE);
    std::vector<__half> whi((size_t)v.Vr * v.Vp), wlo((size_t)v.Vr * v.Vp);
    for (int r = 0; r < v.Vr; ++r)
        for (int k = 0; k < v.Vp; ++k) {
            const double e = (r < V && k < V) ? E[(size_t)r * V + k] * es : 0.0;
            const __half h = __float2half_rn((float)e);
            whi[(size_t)r * v.Vp + k] = h;
            wlo[(size_t)r * v.Vp + k] = __float2half_rn((float)(e - (double)__half2float(h)));
        }
    v.e_inv = (float)std::ldexp(1.0, -eE);
    bool ok = true;
    const size_t N = (size_t)v.N;
    void* dhi = dev_alloc(c, hi.size() * sizeof(__half), &ok);
    void* dlo = dev_alloc(c, lo.size() * sizeof(__half), &ok);
    void* dwhi = dev_alloc(c, whi.size() * sizeof(__half), &ok);
    void* dwlo = dev_alloc(c, wlo.size() * sizeof(__half), &ok);
    v.cis_f = (float2*)dev_alloc(c, N * sizeof(float2), &ok);
    v.r_f = (float2*)dev_alloc(c, N * sizeof(float2), &ok);
    v.p_f = (float2*)dev_alloc(c, N * sizeof(float2), &ok);
    v.p2_f = (float2*)dev_alloc(c, N * sizeof(float2), &ok);
    v.q_f = (float2*)dev_alloc(c, N * sizeof(float2), &ok);
    v.x_f = (float2*)dev_alloc(c, N * sizeof(float2), &ok);
    v.g_f = (float2*)dev_alloc(c, N * sizeof(float2), &ok);
    const size_t Nh = (size_t)(v.Nt + 2) * v.V;   // split-K sources with the halo rows
    v.u_f = (float2*)dev_alloc(c, Nh * sizeof(float2), &ok);
    v.rh_f = (float2*)dev_alloc(c, Nh * sizeof(float2), &ok);
    v.sk_b16 = nullptr;
    v.sk_maps = nullptr;
    v.gslots = (unsigned long long*)dev_alloc(c, tc::kGatherSlots * sizeof(unsigned long long),
                                              &ok);
    if (!ok) return HMC_ERR_CUDA;
    if (cudaMemcpy(dhi, hi.data(), hi.size() * sizeof(__half), cudaMemcpyHostToDevice) !=
            cudaSuccess ||
        cudaMemcpy(dlo, lo.data(), lo.size() * sizeof(__half), cudaMemcpyHostToDevice) !=
            cudaSuccess ||
        cudaMemcpy(dwhi, whi.data(), whi.size() * sizeof(__half), cudaMemcpyHostToDevice) !=
            cudaSuccess ||
        cudaMemcpy(dwlo, wlo.data(), wlo.size() * sizeof(__half), cudaMemcpyHostToDevice) !=
            cudaSuccess)
        return HMC_ERR_CUDA;
    v.E_hi = dhi;
    v.E_lo = dlo;
    v.Ew_hi = dwhi;
    v.Ew_lo = dwlo;
    c->tc = new TcCtx();
    if (!make_map(&c->tc->map_hi, dhi, v.Vr, v.Vp) || !make_map(&c->tc->map_lo, dlo, v.Vr, v.Vp) ||
        !make_map(&c->tc->map_shi, dwhi, v.Vr, v.Vp) || !make_map(&c->tc->map_slo, dwlo, v.Vr, v.Vp))
        return HMC_ERR_CUDA;
    {
        // slice-major tiles: all sites in one tile up to 288; standalone
        // applications above 256 sites take tiles of 144 (one instruction,
        // same TMA box) and as many slice tiles as fill one wave
        TcCtx* t = c->tc;
        t->w_cg = tc::wide_sites(V);
        const tc::WideGeom g = tc::wide_geom(t->w_cg);
        const int box = t->w_cg / g.nmma;
        t->w_apply = V > tc::kWMaxN ? box : t->w_cg;
        // standalone tiles of up to 64 slices (balanced); each tile's K is
        // split over a cluster of up to 8 CTAs while the tiles x split fill
        // the GPU (at least one K chunk per CTA)
        const int nsi = (V + t->w_apply - 1) / t->w_apply;
        const int ntt = (v.Nt + tc::kWSlices - 1) / tc::kWSlices;
        t->ns_wapply = (v.Nt + ntt - 1) / ntt;
        if (c->params.operand_mode == 4 && c->params.tile_slices > 0)
            t->ns_wapply = c->params.tile_slices;
        const int tiles = nsi * ((v.Nt + t->ns_wapply - 1) / t->ns_wapply);
        t->csplit_apply = std::max(1, std::min(std::min(tc::kMaxClusterW, v.Vp / tc::KCH),
                                               c->num_sms / std::max(1, tiles)));
        if (!make_map(&t->map_whi, dwhi, v.Vr, v.Vp, box) ||
            !make_map(&t->map_wlo, dwlo, v.Vr, v.Vp, box))
            return HMC_ERR_CUDA;
    }
    c->tc->ns_apply = pick_ns(v.Vr / tc::TM, v.Nt, c->num_sms);
    if (c->params.tile_slices > 0 && c->params.operand_mode != 4 && c->params.operand_mode != 5)
        c->tc->ns_apply = c->params.tile_slices;
    {
        // pre-split B of standalone applications (rows padded by 64 zero rows)
        const int nb = ((2 * c->tc->ns_apply + 15) / 16) * 16;   // MMA N = TMA box rows
        c->tc->b_rows = 2 * v.Nt + 128;   // a 128-row box from any 2t stays inside
        const size_t nbh = (size_t)c->tc->b_rows * v.Vp;
        bool okb = true;
        c->tc->bhi = (__half*)dev_alloc(c, nbh * sizeof(__half), &okb);
        c->tc->blo = (__half*)dev_alloc(c, nbh * sizeof(__half), &okb);
        c->tc->inv_col = (float*)dev_alloc(c, (size_t)v.Nt * sizeof(float), &okb);
        if (!okb || !make_map(&c->tc->map_bhi, c->tc->bhi, c->tc->b_rows, v.Vp, nb) ||
            !make_map(&c->tc->map_blo, c->tc->blo, c->tc->b_rows, v.Vp, nb) ||
            !make_map(&c->tc->map_uhi, c->tc->bhi, c->tc->b_rows, v.Vp,
                      tc::wide_u_rows(c->tc->ns_wapply)) ||
            !make_map(&c->tc->map_ulo, c->tc->blo, c->tc->b_rows, v.Vp,
                      tc::wide_u_rows(c->tc->ns_wapply)))
            return HMC_ERR_CUDA;
        // split-K standalone applications (operand_mode 5)
        c->tc->sk_C_apply = 0;
        c->tc->sk_ns_apply = 0;
        int skC = 0, skns = 0;
        if (c->params.operand_mode == 5 && splitk_shape(c, &skC, &skns)) {
            if (!make_map(&c->tc->map_skb_hi, c->tc->bhi, c->tc->b_rows, v.Vp, tc::sk_nn(skns)) ||
                !make_map(&c->tc->map_skb_lo, c->tc->blo, c->tc->b_rows, v.Vp, tc::sk_nn(skns)))
                return HMC_ERR_CUDA;
            c->tc->sk_C_apply = skC;
            c->tc->sk_ns_apply = skns;
            c->tc->inv_sk = (float*)dev_alloc(c, (size_t)v.Nt * skC * sizeof(float), &okb);
            if (!okb) return HMC_ERR_CUDA;
            // the CG's sources: r and u with their halo rows, boxes of ns rows,
            // and their FP16 splits, boxes of sk_nn(ns) rows
            const int rows16 = 2 * (v.Nt + 2);
            const size_t plane = (size_t)rows16 * v.Vp;
            __half_raw* b16 = (__half_raw*)dev_alloc(c, 4 * plane * sizeof(__half), &okb);
            if (!okb) return HMC_ERR_CUDA;
            c->view.sk_b16 = b16;
            CUtensorMap hm[6];
            if (!make_map_src(&hm[0], c->view.rh_f, v.Nt + 2, V, skns) ||
                !make_map_src(&hm[1], c->view.u_f, v.Nt + 2, V, skns))
                return HMC_ERR_CUDA;
            for (int q = 0; q < 4; ++q)
                if (!make_map(&hm[2 + q], b16 + q * plane, rows16, v.Vp, tc::sk_nn(skns)))
                    return HMC_ERR_CUDA;
            void* dm = dev_alloc(c, sizeof(hm), &okb);
            if (!okb || cudaMemcpy(dm, hm, sizeof(hm), cudaMemcpyHostToDevice) != cudaSuccess)
                return HMC_ERR_CUDA;
            c->view.sk_maps = dm;
        }
        const int split_smem = V * (int)sizeof(float2);
        for (const void* k : {(const void*)tc::k_split<false, false>,
                              (const void*)tc::k_split<true, false>,
                              (const void*)tc::k_split<false, true>,
                              (const void*)tc::k_split<true, true>})
            if (split_smem > 48 * 1024 &&
                cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     split_smem) != cudaSuccess)
                return HMC_ERR_CUDA;
    }
    const void* kernels[] = {(const void*)tc::k_apply<false>,
                             (const void*)tc::k_apply<true>,
                             (const void*)tc::k_apply_sk<false>,
                             (const void*)tc::k_apply_sk<true>,
                             (const void*)tc::k_apply_w<false>,
                             (const void*)tc::k_apply_w<true>,
                             (const void*)tc::k_cg<tc::kKindSite>,
                             (const void*)tc::k_trajectory<tc::kKindSite>,
                             (const void*)tc::k_cg<tc::kKindSmall>,
                             (const void*)tc::k_trajectory<tc::kKindSmall>,
                             (const void*)tc::k_cg<tc::kKindSlice>,
                             (const void*)tc::k_trajectory<tc::kKindSlice>,
                             (const void*)tc::k_cg<tc::kKindSplitK>,
                             (const void*)tc::k_trajectory<tc::kKindSplitK>};
    for (const void* k : kernels)
        if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)tc::kSmemBytes) != cudaSuccess)
            return HMC_ERR_CUDA;
    // the small-lattice mode may run on clusters of up to 16 CTAs (beyond the
    // portable 8); a device that cannot co-schedule them refuses the launch
    for (const void* k : {(const void*)tc::k_cg<tc::kKindSmall>,
                          (const void*)tc::k_trajectory<tc::kKindSmall>})
        if (cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
            cudaSuccess)
            (void)cudaGetLastError();
    return HMC_OK;
}

void tc_ctx_free(hmc_ctx* c) {
    delete c->tc;
    c->tc = nullptr;
}

// Launch an application kernel as a programmatic dependent of the split
// that precedes it on the stream (its set-up overlaps the split; it waits
// with griddepcontrol.wait before reading the split's output), in clusters
// of `cluster` CTAs when cluster > 1.
static int launch_dependent(const void* fn, int grid, int cluster, void** args,
                            cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(tc::NTHR);
    cfg.dynamicSmemBytes = tc::kSmemBytes;
    cfg.stream = s;
    cudaLaunchAttribute at[2];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    at[1].id = cudaLaunchAttributeClusterDimension;
    at[1].val.clusterDim.x = (unsigned)cluster;
    at[1].val.clusterDim.y = 1;
    at[1].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = cluster > 1 ? 2 : 1;
    return cudaLaunchKernelExC(&cfg, fn, args) == cudaSuccess ? HMC_OK : HMC_ERR_CUDA;
}

int tc_apply(hmc_ctx* c, const double* phi, const float2* in, float2* out, bool dag,
             cudaStream_t s) {
    const ChainView& v = c->view;
    const size_t split_smem = (size_t)v.V * sizeof(float2);
    TcCtx* t = c->tc;
    if (c->params.operand_mode == 5 && t->sk_C_apply > 0) {
        int C = t->sk_C_apply, ns = t->sk_ns_apply;
        const int grid = (v.Vr / tc::TM) * ((v.Nt + ns - 1) / ns) * C;
        const dim3 sgrid(v.Nt, C);
        if (dag)
            tc::k_split_sk<true><<<sgrid, tc::kSplitSkThreads, 0, s>>>(
                phi, in, v.cis_f, t->bhi, t->blo, t->inv_sk, v.V, v.Vp, v.Nt, C);
        else
            tc::k_split_sk<false><<<sgrid, tc::kSplitSkThreads, 0, s>>>(
                phi, in, v.cis_f, t->bhi, t->blo, t->inv_sk, v.V, v.Vp, v.Nt, C);
        if (cudaGetLastError() != cudaSuccess) return HMC_ERR_CUDA;
        ChainView vv = v;
        const float2* inp = in;
        float2* outp = out;
        const float* invp = t->inv_sk;
        void* args[] = {&t->map_shi, &t->map_slo, &t->map_skb_hi, &t->map_skb_lo, &vv,
                        &C, &ns, &inp, &outp, &invp};
        return launch_dependent(
            dag ? (const void*)tc::k_apply_sk<true> : (const void*)tc::k_apply_sk<false>, grid,
            C, args, s);
    }
    if (c->params.operand_mode == 4) {
        int W = t->w_apply, ns = t->ns_wapply, cs = t->csplit_apply;
        const int tiles = ((v.V + W - 1) / W) * ((v.Nt + ns - 1) / ns);
        if (dag)
            tc::k_split<true, true><<<v.Nt, tc::kSplitThreads, split_smem, s>>>(
                phi, in, v.cis_f, t->bhi, t->blo, t->inv_col, v.V, v.Vp, v.Nt);
        else
            tc::k_split<false, true><<<v.Nt, tc::kSplitThreads, split_smem, s>>>(
                phi, in, v.cis_f, t->bhi, t->blo, t->inv_col, v.V, v.Vp, v.Nt);
        if (cudaGetLastError() != cudaSuccess) return HMC_ERR_CUDA;
        ChainView vv = v;
        const float2* inp = in;
        float2* outp = out;
        const float* invp = t->inv_col;
        void* args[] = {&t->map_whi, &t->map_wlo, &t->map_uhi, &t->map_ulo, &vv,
                        &W, &ns, &cs, &inp, &outp, &invp};
        return launch_dependent(
            dag ? (const void*)tc::k_apply_w<true> : (const void*)tc::k_apply_w<false>,
            tiles * cs, cs, args, s);
    }
    int ns = c->tc->ns_apply;
    const int tiles = (v.Vr / tc::TM) * ((v.Nt + ns - 1) / ns);
    if (dag)
        tc::k_split<true, false><<<v.Nt, tc::kSplitThreads, split_smem, s>>>(
            phi, in, v.cis_f, t->bhi, t->blo, t->inv_col, v.V, v.Vp, v.Nt);
    else
        tc::k_split<false, false><<<v.Nt, tc::kSplitThreads, split_smem, s>>>(
            phi, in, v.cis_f, t->bhi, t->blo, t->inv_col, v.V, v.Vp, v.Nt);
    if (cudaGetLastError() != cudaSuccess) return HMC_ERR_CUDA;
    ChainView vv = v;
    const float2* inp = in;
    float2* outp = out;
    const float* invp = t->inv_col;
    void* args[] = {&t->map_hi, &t->map_lo, &t->map_bhi, &t->map_blo, &vv, &ns, &inp, &outp, &invp};
    return launch_dependent(dag ? (const void*)tc::k_apply<true> : (const void*)tc::k_apply<false>,
                            tiles, 1, args, s);
}

static int team_size(hmc_ctx* c, const void* kernel) {
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, tc::NTHR, tc::kSmemBytes) !=
            cudaSuccess ||
        occ < 1)
        return -1;
    const ChainView& v = c->view;
    const int f64_tiles = ((v.V + f64::TI - 1) / f64::TI) * ((v.Nt + f64::TT - 1) / f64::TT);
    const int tc_tiles = (v.Vr / tc::TM) * ((v.Nt + 7) / 8);
    int want = std::max(f64_tiles, tc_tiles);
    if (c->params.team_ctas > 0) want = c->params.team_ctas;
    int g = std::min(c->num_sms * occ, kMaxTeam);
    return std::max(1, std::min(g, want));
}

// Resident B per slice tile pays when a CTA runs several site blocks of the
// same slices: streaming layout, at least two site blocks, every CTA of the
// inner team with a slice tile, and the tile's B within the area after the
// E ring.
static bool res_b_ok(const ChainView& v, int mode, int ns, int inner) {
    const int nti = v.Vr / tc::TM, ntt = (v.Nt + ns - 1) / ns;
    const int N = ((2 * ns + 15) / 16) * 16;
    return mode == tc::kStreaming && nti >= 2 && inner <= ntt &&
           tc::res_b_bytes(N, v.Vp) <= tc::kResBArea;
}

// Cluster size of the small-lattice CUDA-core mode: inner_ctas when given,
// else the largest of 8, 4, 2, 1 that fits (each CTA at least 2 slices).
static int small_cluster(const hmc_ctx* c) {
    const ChainView& v = c->view;
    if (c->params.inner_ctas > 0)
        return tc::small_feasible(v.V, v.Nt, c->params.inner_ctas) ? c->params.inner_ctas : 0;
    for (int C = 16; C >= 1; C >>= 1)
        if ((C == 1 || v.Nt >= 2 * C) && tc::small_feasible(v.V, v.Nt, C)) return C;
    return 0;
}

// Split-K shape (operand_mode 5): slices per n-group (tile_slices, else the
// fewest n-groups of at most 64 slices, balanced) and CTAs per cluster
// (inner_ctas, else the smallest of 6, 8, 4, 2 whose K range fits the
// shared memory); false if the requested shape does not fit.
static bool splitk_shape(const hmc_ctx* c, int* C_out, int* ns_out) {
    const ChainView& v = c->view;
    int ns = c->params.tile_slices;
    if (ns <= 0) {
        const int nng = (v.Nt + 63) / 64;
        ns = (v.Nt + nng - 1) / nng;
    }
    if (ns < 1 || ns > 64) return false;
    const int Nn = tc::sk_nn(ns);
    const int KS = (v.V + 15) / 16;
    auto fits = [&](int C) {
        if (C < 2 || C > tc::kSkMaxCluster || C > KS) return false;
        const int steps = (KS + C - 1) / C;
        const int nch = tc::sk_chunks(steps);
        const int own_slices = (std::min(ns, v.Nt) + C - 1) / C;
        return nch <= tc::kSkMaxChunks &&
               tc::sk_smem_total(nch, Nn, own_slices) <= tc::kOperandBytes;
    };
    int C = c->params.inner_ctas;
    if (C > 0) {
        if (!fits(C)) return false;
    } else {
        C = 0;
        for (int cand : {6, 8, 4, 2})
            if (fits(cand)) { C = cand; break; }
        if (!C) return false;
    }
    *C_out = C;
    *ns_out = ns;
    return true;
}

static tc::PersistentArgs persistent_args(hmc_ctx* c, int grid, double tol, int max_iter) {
    tc::PersistentArgs pa;
    const ChainView& v = c->view;
    pa.sk_C = 0;
    if (c->params.operand_mode == 5) {
        // split-K tiles with E' resident: nib x nng clusters of C CTAs form
        // the inner team (0 CTAs if the shape does not fit)
        int C = 0, ns = 0;
        pa.mode = tc::kSplitK;
        pa.inner = 0;
        if (splitk_shape(c, &C, &ns)) {
            pa.sk_C = C;
            pa.ns_tile = ns;
            pa.inner = (v.Vr / tc::TM) * ((v.Nt + ns - 1) / ns) * C;
        }
        pa.cluster = C;
        pa.vec_resident = 0;
        pa.res_b = 0;
        pa.wide_W = 0;
        pa.tol = tol;
        pa.max_iter = max_iter;
        pa.ru_delta = c->params.ru_delta;
        pa.ru_every = c->params.ru_every;
        (void)grid;
        return pa;
    }
    if (c->params.operand_mode == 3) {
        // CUDA-core cluster solver; grid is a multiple of the cluster size
        pa.mode = tc::kSmall;
        pa.inner = small_cluster(c);
        pa.ns_tile = 8;
        pa.vec_resident = 0;
        pa.tol = tol;
        pa.max_iter = max_iter;
        pa.ru_delta = c->params.ru_delta;
        pa.ru_every = c->params.ru_every;
        pa.cluster = 0;
        pa.res_b = 0;
        pa.wide_W = 0;
        return pa;
    }
    pa.wide_W = 0;
    if (c->params.operand_mode == 4) {
        // slice-major tiles: one CTA per tile at 64 slices by default
        pa.mode = tc::kSlice;
        pa.wide_W = c->tc->w_cg;
        const int ntt64 = (v.Nt + tc::kWSlices - 1) / tc::kWSlices;
        pa.inner = std::min(grid, ((v.V + pa.wide_W - 1) / pa.wide_W) * ntt64);
        if (c->params.inner_ctas > 0) pa.inner = std::min(c->params.inner_ctas, grid);
        const int nsi = (v.V + pa.wide_W - 1) / pa.wide_W;
        // slices per tile: balanced over enough slice tiles for the team
        const int want_tt = std::max(ntt64, (pa.inner + nsi - 1) / nsi);
        pa.ns_tile = std::min(tc::kWSlices, (v.Nt + want_tt - 1) / want_tt);
        if (c->params.tile_slices > 0) pa.ns_tile = c->params.tile_slices;
        pa.vec_resident = 0;
        pa.tol = tol;
        pa.max_iter = max_iter;
        pa.ru_delta = c->params.ru_delta;
        pa.ru_every = c->params.ru_every;
        pa.cluster = 0;
        pa.res_b = 0;
        return pa;
    }
    // inner team: one CTA while the whole lattice fits in a handful of tiles
    // (a single CTA needs no inter-CTA barrier), else the whole launch
    const int nti = v.Vr / tc::TM;
    const int nk = v.Vp / tc::KCH;
    // resident E when one site block's rows (all K) fit and every site block
    // gets its own CTA; else stream E through the ring
    const bool can_resident = nk <= tc::kMaxResidentChunks && nti <= grid;
    pa.mode = (c->params.operand_mode == 2 || (c->params.operand_mode == 0 && can_resident))
                  ? tc::kResident
                  : tc::kStreaming;
    if (pa.mode == tc::kResident && !can_resident) pa.mode = tc::kStreaming;
    pa.vec_resident = 0;
    if (pa.mode == tc::kResident) {
        // one CTA per site block, or (inner_ctas) a multiple of that: the
        // extra CTAs take further slice tiles of the same block
        pa.inner = nti;
        if (c->params.inner_ctas > nti)
            pa.inner = std::min(c->params.inner_ctas / nti, grid / nti) * nti;
        pa.ns_tile = std::min(16, pick_ns(1, v.Nt, pa.inner / nti));
        const size_t free_bytes =
            tc::kOperandBytes - (size_t)nk * tc::kAChunkBytes - tc::kMaxStages * tc::kBStageSmall;
        pa.vec_resident =
            (pa.inner == 1 && 6 * sizeof(float2) * (size_t)v.N <= free_bytes) ? 1 : 0;
    } else {
        pa.inner = nti * ((v.Nt + 31) / 32) <= 2 ? 1 : grid;
        if (c->params.inner_ctas > 0) pa.inner = std::min(c->params.inner_ctas, grid);
        pa.ns_tile = pick_ns(nti, v.Nt, pa.inner);
    }
    if (c->params.tile_slices > 0) pa.ns_tile = c->params.tile_slices;
    if (pa.mode == tc::kResident && pa.ns_tile > 16) pa.ns_tile = 16;   // 8 KB B stages
    pa.tol = tol;
    pa.max_iter = max_iter;
    pa.ru_delta = c->params.ru_delta;
    pa.ru_every = c->params.ru_every;
    pa.cluster = 0;
    pa.res_b = res_b_ok(v, pa.mode, pa.ns_tile, pa.inner) ? 1 : 0;
    return pa;
}

// Cooperative launch of a persistent kernel.  An inner team of 2..8 CTAs
// that divides the grid is launched as thread-block clusters (cluster 0 is
// the inner team) unless cluster_mode says never; in automatic mode a
// refused cluster launch falls back to global-memory team barriers.
// `pa` is the object args points at.
static int launch_persistent(hmc_ctx* c, const void* fn, int grid, void** args,
                             tc::PersistentArgs& pa, cudaStream_t s) {
    int cm = c->params.cluster_mode;
    if (pa.mode == tc::kSmall) {
        // the small mode reads its peers' shared memory: a cluster or nothing
        if (pa.inner < 1 || grid % pa.inner != 0) return HMC_ERR_UNSUPPORTED;
        if (pa.inner > 1) {
            if (cm == 2) return HMC_ERR_UNSUPPORTED;
            cm = 1;
        }
    }
    const int max_cluster = pa.mode == tc::kSmall ? tc::kSmallMaxCluster : 8;
    const bool want = cm != 2 && pa.inner > 1 && pa.inner <= max_cluster && grid % pa.inner == 0;
    if (cm == 1 && !want) return HMC_ERR_UNSUPPORTED;
    if (want) {
        pa.cluster = pa.inner;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(grid);
        cfg.blockDim = dim3(tc::NTHR);
        cfg.dynamicSmemBytes = tc::kSmemBytes;
        cfg.stream = s;
        // the CTAs of one cluster are scheduled together, so a launch that
        // is one cluster needs no cooperative attribute; several clusters
        // take it for the team barriers between them
        cudaLaunchAttribute at[2];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = (unsigned)pa.inner;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        at[1].id = cudaLaunchAttributeCooperative;
        at[1].val.cooperative = 1;
        cfg.attrs = at;
        cfg.numAttrs = grid == pa.inner ? 1 : 2;
        if (cudaLaunchKernelExC(&cfg, fn, args) == cudaSuccess) return HMC_OK;
        (void)cudaGetLastError();   // a refused configuration is not sticky
        pa.cluster = 0;
        if (cm == 1) return HMC_ERR_UNSUPPORTED;
    }
    return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(tc::NTHR), args, tc::kSmemBytes, s) ==
                   cudaSuccess
               ? HMC_OK
               : HMC_ERR_CUDA;
}

// Split-K mode: a cooperative launch of thread-block clusters of sk_C CTAs,
// as many clusters as can be resident at once (at least the inner team's;
// team_ctas caps it), with the team-sum slots cleared first.
static int launch_splitk(hmc_ctx* c, const void* fn, void** args, tc::PersistentArgs& pa,
                         cudaStream_t s) {
    if (pa.inner < 1 || pa.sk_C < 2) return HMC_ERR_UNSUPPORTED;
    cudaLaunchConfig_t cfg = {};
    cfg.blockDim = dim3(tc::NTHR);
    cfg.dynamicSmemBytes = tc::kSmemBytes;
    cfg.stream = s;
    cudaLaunchAttribute at[2];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)pa.sk_C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    at[1].id = cudaLaunchAttributeCooperative;
    at[1].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cfg.gridDim = dim3(pa.inner);
    int nclu = 0;
    if (cudaOccupancyMaxActiveClusters(&nclu, fn, &cfg) != cudaSuccess) {
        (void)cudaGetLastError();
        return HMC_ERR_UNSUPPORTED;
    }
    int grid = std::min(nclu * pa.sk_C, kMaxTeam / pa.sk_C * pa.sk_C);
    if (c->params.team_ctas > 0)
        grid = std::min(grid, std::max(c->params.team_ctas / pa.sk_C * pa.sk_C, pa.inner));
    if (grid < pa.inner) return HMC_ERR_UNSUPPORTED;
    cfg.gridDim = dim3(grid);
    // HMC_PROFILE_NONCOOPERATIVE=1: the same launch without the cooperative
    // attribute, for profilers that refuse cooperative cluster launches.  The
    // grid is the clusters that can be resident at once, so in practice every
    // CTA runs; were one not resident, the bounded team waits would end the
    // launch with HMC_ERR_TIMEOUT.
    cfg.numAttrs = getenv("HMC_PROFILE_NONCOOPERATIVE") ? 1 : 2;
    if (cudaMemsetAsync(c->view.gslots, 0, tc::kGatherSlots * sizeof(unsigned long long), s) !=
        cudaSuccess)
        return HMC_ERR_CUDA;
    pa.cluster = pa.sk_C;
    if (cudaLaunchKernelExC(&cfg, fn, args) != cudaSuccess) {
        (void)cudaGetLastError();
        return HMC_ERR_UNSUPPORTED;
    }
    return HMC_OK;
}

// Small mode: the launch is a whole number of clusters.
static int round_grid(const tc::PersistentArgs& pa, int grid) {
    if (pa.mode != tc::kSmall || pa.inner < 1) return grid;
    return std::max(pa.inner, grid / pa.inner * pa.inner);
}

int tc_cg(hmc_ctx* c, const double* phi, const double2* chi, double2* x, double tol,
          int max_iter, cudaStream_t s) {
    int grid = team_size(c, (const void*)tc::k_cg<tc::kKindSite>);
    if (grid < 1) return HMC_ERR_CUDA;
    tc::PersistentArgs pa = persistent_args(c, grid, tol, max_iter);
    if (pa.mode == tc::kSmall && pa.inner < 1) return HMC_ERR_UNSUPPORTED;
    grid = round_grid(pa, grid);
    ChainView v = c->view;
    if (pa.mode == tc::kSplitK) {
        void* args[] = {&c->tc->map_shi, &c->tc->map_slo, &v, &pa, &phi, &chi, &x};
        return launch_splitk(c, (const void*)tc::k_cg<tc::kKindSplitK>, args, pa, s);
    }
    const void* fn = pa.mode == tc::kSmall   ? (const void*)tc::k_cg<tc::kKindSmall>
                     : pa.mode == tc::kSlice ? (const void*)tc::k_cg<tc::kKindSlice>
                                             : (const void*)tc::k_cg<tc::kKindSite>;
    const bool sl = pa.mode == tc::kSlice;
    void* args[] = {sl ? &c->tc->map_whi : &c->tc->map_hi, sl ? &c->tc->map_wlo : &c->tc->map_lo,
                    &v, &pa, &phi, &chi, &x};
    return launch_persistent(c, fn, grid, args, pa, s);
}

int tc_trajectory(hmc_ctx* c, const TrajArgs& a, cudaStream_t s) {
    int grid = team_size(c, (const void*)tc::k_trajectory<tc::kKindSite>);
    if (grid < 1) return HMC_ERR_CUDA;
    tc::PersistentArgs pa = persistent_args(c, grid, a.tol, a.max_iter);
    if (pa.mode == tc::kSmall && pa.inner < 1) return HMC_ERR_UNSUPPORTED;
    grid = round_grid(pa, grid);
    ChainView v = c->view;
    TrajArgs av = a;
    if (pa.mode == tc::kSplitK) {
        void* args[] = {&c->tc->map_shi, &c->tc->map_slo, &v, &pa, &av};
        return launch_splitk(c, (const void*)tc::k_trajectory<tc::kKindSplitK>, args, pa, s);
    }
    const void* fn = pa.mode == tc::kSmall   ? (const void*)tc::k_trajectory<tc::kKindSmall>
                     : pa.mode == tc::kSlice ? (const void*)tc::k_trajectory<tc::kKindSlice>
                                             : (const void*)tc::k_trajectory<tc::kKindSite>;
    const bool sl = pa.mode == tc::kSlice;
    void* args[] = {sl ? &c->tc->map_whi : &c->tc->map_hi, sl ? &c->tc->map_wlo : &c->tc->map_lo,
                    &v, &pa, &av};
    return launch_persistent(c, fn, grid, args, pa, s);
}


// ---------------------------------------------------------------- batch (host)
struct TcBatch {
    int n = 0;
    int grid = 0;
    int csize = 1;                   // CTAs per cluster (> 1: team chains present)
    std::vector<hmc_ctx*> ctxs;
    std::vector<long long> offsets;   // n + 1
    tc::BatchItem* d_items = nullptr;
    int* d_order = nullptr;
    int* d_queue = nullptr;
    tc::BatchCallArgs* d_call = nullptr;
    tc::BatchCallArgs* h_call = nullptr;   // pinned
    double* d_outs = nullptr;
    double* h_outs = nullptr;          // pinned
    CUtensorMap* d_maps = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t ready = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    double* graph_phi = nullptr;
};

void tc_batch_destroy(TcBatch* b) {
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->ready) cudaEventDestroy(b->ready);
    if (b->stream) cudaStreamDestroy(b->stream);
    cudaFree(b->d_items);
    cudaFree(b->d_order);
    cudaFree(b->d_queue);
    cudaFree(b->d_call);
    cudaFree(b->d_outs);
    cudaFree(b->d_maps);
    if (b->h_call) cudaFreeHost(b->h_call);
    if (b->h_outs) cudaFreeHost(b->h_outs);
    for (hmc_ctx* c : b->ctxs) hmc_ctx_destroy(c);
    delete b;
}

int tc_batch_create(const hmc_params* p, int n, TcBatch** out) {
    TcBatch* b = new TcBatch();
    b->n = n;
    int st = HMC_OK;
    // one context per chain (workspaces); chains with the same lattice,
    // delta*kappa and delta*mu share the first such context's E, its splits
    // and maps
    std::vector<int> leader(n);
    std::vector<int> map_slot(n);
    int n_maps = 0;
    for (int i = 0; i < n && st == HMC_OK; ++i) {
        if (p[i].precision != HMC_PREC_MIXED || p[i].operand_mode == 5) st = HMC_ERR_UNSUPPORTED;
        hmc_ctx* c = nullptr;
        if (st == HMC_OK) st = hmc_ctx_create(&p[i], &c);
        if (st != HMC_OK) break;
        b->ctxs.push_back(c);
        leader[i] = i;
        for (int j = 0; j < i; ++j)
            if (p[j].L == p[i].L &&
                p[j].beta / p[j].Nt * p[j].kappa == p[i].beta / p[i].Nt * p[i].kappa &&
                p[j].beta / p[j].Nt * p[j].mu == p[i].beta / p[i].Nt * p[i].mu) {
                leader[i] = leader[j];
                break;
            }
        map_slot[i] = (leader[i] == i) ? n_maps++ : map_slot[leader[i]];
    }
    if (st != HMC_OK) {
        tc_batch_destroy(b);
        return st;
    }
    std::vector<CUtensorMap> maps(4 * n_maps);
    for (int i = 0; i < n; ++i)
        if (leader[i] == i) {
            maps[4 * map_slot[i]] = b->ctxs[i]->tc->map_hi;
            maps[4 * map_slot[i] + 1] = b->ctxs[i]->tc->map_lo;
            maps[4 * map_slot[i] + 2] = b->ctxs[i]->tc->map_whi;
            maps[4 * map_slot[i] + 3] = b->ctxs[i]->tc->map_wlo;
        }
    // chains asking for a team (team_ctas >= 2) run on a thread-block
    // cluster of that many CTAs; all such chains of a batch use one size
    for (int i = 0; i < n; ++i) {
        const int tmc = p[i].team_ctas;
        if (tmc <= 1) continue;
        if (tmc > tc::kMaxClusterW || (b->csize > 1 && tmc != b->csize)) {
            tc_batch_destroy(b);
            return HMC_ERR_UNSUPPORTED;
        }
        b->csize = tmc;
    }
    std::vector<tc::BatchItem> items(n);
    b->offsets.assign(n + 1, 0);
    std::vector<double> cost(n);
    for (int i = 0; i < n; ++i) {
        hmc_ctx* c = b->ctxs[i];
        const ChainView& lv = b->ctxs[leader[i]]->view;
        tc::BatchItem& it = items[i];
        it.v = c->view;
        it.v.E = lv.E;
        it.v.E_hi = lv.E_hi;
        it.v.E_lo = lv.E_lo;
        it.v.Ew_hi = lv.Ew_hi;
        it.v.Ew_lo = lv.Ew_lo;
        it.v.e_inv = lv.e_inv;
        it.team = c->params.team_ctas > 1 ? c->params.team_ctas : 1;
        it.pa.inner = 1;
        it.pa.cluster = 0;
        if (it.team > 1) {
            // a cluster team: the launch shape of a single-chain run on
            // team CTAs with an inner team of all of them, as one cluster
            if (c->params.inner_ctas == 0) c->params.inner_ctas = it.team;
            it.pa = persistent_args(c, it.team, c->params.cg_tol, c->params.cg_max_iter);
            if (it.pa.inner != it.team || (it.pa.mode == tc::kSmall && it.pa.inner < 1)) {
                tc_batch_destroy(b);
                return HMC_ERR_UNSUPPORTED;
            }
            it.pa.cluster = it.team;
        } else {
            // one CTA per chain: E resident when the chain has one site block
            const int nti = it.v.Vr / tc::TM, nk = it.v.Vp / tc::KCH;
            const bool res = nti == 1 && nk <= tc::kMaxResidentChunks &&
                             c->params.operand_mode != 1;
            it.pa.mode = res ? tc::kResident : tc::kStreaming;
            it.pa.ns_tile = pick_ns(nti, it.v.Nt, 1);
            if (c->params.tile_slices > 0) it.pa.ns_tile = c->params.tile_slices;
            it.pa.vec_resident = 0;
            if (res) {
                it.pa.ns_tile = std::min(it.pa.ns_tile, 16);
                const size_t free_bytes = tc::kOperandBytes - (size_t)nk * tc::kAChunkBytes -
                                          tc::kMaxStages * tc::kBStageSmall;
                it.pa.vec_resident = 6 * sizeof(float2) * (size_t)it.v.N <= free_bytes;
            }
            // operand_mode 3: the CUDA-core solver on the chain's one CTA
            if (c->params.operand_mode == 3 && tc::small_feasible(it.v.V, it.v.Nt, 1)) {
                it.pa.mode = tc::kSmall;
                it.pa.vec_resident = 0;
            }
            it.pa.res_b = res_b_ok(it.v, it.pa.mode, it.pa.ns_tile, 1) ? 1 : 0;
            it.pa.wide_W = 0;
            // operand_mode 4: slice-major tiles, balanced slices of at most 64
            if (c->params.operand_mode == 4) {
                it.pa.mode = tc::kSlice;
                it.pa.wide_W = c->tc->w_cg;
                const int ntt = (it.v.Nt + tc::kWSlices - 1) / tc::kWSlices;
                it.pa.ns_tile = (it.v.Nt + ntt - 1) / ntt;
                if (c->params.tile_slices > 0) it.pa.ns_tile = c->params.tile_slices;
                it.pa.res_b = 0;
                it.pa.vec_resident = 0;
            }
        }
        if (it.team > 1) it.pa.res_b = 0;
        it.pa.tol = c->params.cg_tol;
        it.pa.max_iter = c->params.cg_max_iter;
        it.pa.ru_delta = c->params.ru_delta;
        it.pa.ru_every = c->params.ru_every;
        std::memset(&it.a, 0, sizeof(it.a));
        it.a.chain = (uint32_t)i;
        it.a.n_md = c->params.n_md;
        it.a.integrator = c->params.integrator;
        it.a.eps = c->params.traj_length / c->params.n_md;
        it.a.tol = c->params.cg_tol;
        it.a.max_iter = c->params.cg_max_iter;
        it.a.ru_delta = c->params.ru_delta;
        it.offset = b->offsets[i];
        b->offsets[i + 1] = b->offsets[i] + it.v.N;
        // cost proxy: tile work of one application times Nt (CG iterations
        // grow with beta = Nt * delta)
        cost[i] = (double)it.v.Vr * it.v.Vp * it.v.Nt * it.v.Nt;
    }
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    // team chains first (the cluster phase of the kernel), then by cost
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) {
        if ((items[a].team > 1) != (items[c].team > 1)) return items[a].team > 1;
        return cost[a] > cost[c];
    });
    bool ok = true;
    auto alloc = [&](void** ptr, size_t bytes) {
        if (ok && cudaMalloc(ptr, bytes) != cudaSuccess) ok = false;
    };
    alloc((void**)&b->d_maps, sizeof(CUtensorMap) * maps.size());
    alloc((void**)&b->d_items, sizeof(tc::BatchItem) * n);
    alloc((void**)&b->d_order, sizeof(int) * n);
    alloc((void**)&b->d_queue, sizeof(int));
    alloc((void**)&b->d_call, sizeof(tc::BatchCallArgs));
    alloc((void**)&b->d_outs, sizeof(double) * kNumScalars * n);
    if (ok && (cudaMallocHost((void**)&b->h_call, sizeof(tc::BatchCallArgs)) != cudaSuccess ||
               cudaMallocHost((void**)&b->h_outs, sizeof(double) * kNumScalars * n) !=
                   cudaSuccess))
        ok = false;
    if (ok) {
        for (int i = 0; i < n; ++i) items[i].maps = b->d_maps + 4 * map_slot[i];
        ok = cudaMemcpy(b->d_maps, maps.data(), sizeof(CUtensorMap) * maps.size(),
                        cudaMemcpyHostToDevice) == cudaSuccess &&
             cudaMemcpy(b->d_items, items.data(), sizeof(tc::BatchItem) * n,
                        cudaMemcpyHostToDevice) == cudaSuccess &&
             cudaMemcpy(b->d_order, order.data(), sizeof(int) * n, cudaMemcpyHostToDevice) ==
                 cudaSuccess &&
             cudaFuncSetAttribute((const void*)tc::k_batch,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)tc::kSmemBytes) == cudaSuccess &&
             cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&b->ready, cudaEventDisableTiming) == cudaSuccess;
    }
    int occ = 0;
    if (ok && (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, (const void*)tc::k_batch,
                                                             tc::NTHR, tc::kSmemBytes) !=
                   cudaSuccess ||
               occ < 1))
        ok = false;
    if (!ok) {
        tc_batch_destroy(b);
        return HMC_ERR_CUDA;
    }
    b->grid = std::min(n, b->ctxs[0]->num_sms * occ);
    if (b->csize > 1) {
        // whole clusters, as many as can be resident at once
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(b->ctxs[0]->num_sms / b->csize * b->csize);
        cfg.blockDim = dim3(tc::NTHR);
        cfg.dynamicSmemBytes = tc::kSmemBytes;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = (unsigned)b->csize;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int nclus = 0;
        if (cudaOccupancyMaxActiveClusters(&nclus, (const void*)tc::k_batch, &cfg) !=
                cudaSuccess ||
            nclus < 1) {
            (void)cudaGetLastError();
            tc_batch_destroy(b);
            return HMC_ERR_UNSUPPORTED;
        }
        b->grid = nclus * b->csize;
    }
    *out = b;
    return HMC_OK;
}

void tc_batch_offsets(const TcBatch* b, long long* off) {
    for (int i = 0; i <= b->n; ++i) off[i] = b->offsets[i];
}

int tc_batch_size(const TcBatch* b) { return b->n; }

// One trajectory of every chain: the launch is captured once into a CUDA
// graph on the batch's own stream (H2D of the call arguments from pinned
// memory, queue reset, the persistent kernel, D2H of the results) and
// replayed; it is ordered after the caller's stream by an event.
int tc_batch_trajectory(TcBatch* b, double* phi, uint64_t seed, uint64_t traj,
                        hmc_traj_out* out, cudaStream_t caller) {
    if (!b->exec || b->graph_phi != phi) {
        if (b->exec) cudaGraphExecDestroy(b->exec);
        if (b->graph) cudaGraphDestroy(b->graph);
        b->exec = nullptr;
        b->graph = nullptr;
        cudaStream_t s = b->stream;
        if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
            return HMC_ERR_CUDA;
        cudaMemcpyAsync(b->d_call, b->h_call, sizeof(tc::BatchCallArgs), cudaMemcpyHostToDevice, s);
        cudaMemsetAsync(b->d_queue, 0, sizeof(int), s);
        {
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(b->grid);
            cfg.blockDim = dim3(tc::NTHR);
            cfg.dynamicSmemBytes = tc::kSmemBytes;
            cfg.stream = s;
            cudaLaunchAttribute at[1];
            at[0].id = cudaLaunchAttributeClusterDimension;
            at[0].val.clusterDim.x = (unsigned)b->csize;
            at[0].val.clusterDim.y = 1;
            at[0].val.clusterDim.z = 1;
            cfg.attrs = at;
            cfg.numAttrs = b->csize > 1 ? 1 : 0;
            const tc::BatchItem* ip = b->d_items;
            const int* op = b->d_order;
            int nn = b->n, cs = b->csize;
            int* qp = b->d_queue;
            const tc::BatchCallArgs* cp = b->d_call;
            double* outp = b->d_outs;
            void* args[] = {&ip, &op, &nn, &qp, &cp, &outp, &cs};
            cudaLaunchKernelExC(&cfg, (const void*)tc::k_batch, args);
        }
        cudaMemcpyAsync(b->h_outs, b->d_outs, sizeof(double) * kNumScalars * b->n,
                        cudaMemcpyDeviceToHost, s);
        if (cudaStreamEndCapture(s, &b->graph) != cudaSuccess ||
            cudaGraphInstantiate(&b->exec, b->graph, 0) != cudaSuccess)
            return HMC_ERR_CUDA;
        b->graph_phi = phi;
    }
    b->h_call->seed = seed;
    b->h_call->traj = traj;
    b->h_call->phi = phi;
    if (cudaEventRecord(b->ready, caller) != cudaSuccess ||
        cudaStreamWaitEvent(b->stream, b->ready, 0) != cudaSuccess ||
        cudaGraphLaunch(b->exec, b->stream) != cudaSuccess ||
        cudaStreamSynchronize(b->stream) != cudaSuccess)
        return HMC_ERR_CUDA;
    int first_bad = HMC_OK;
    for (int i = 0; i < b->n; ++i) {
        const double* v = b->h_outs + (size_t)i * kNumScalars;
        hmc_traj_out& o = out[i];
        o.dH = v[kTrajDH];
        o.H0 = v[kTrajH0];
        o.H1 = v[kTrajH1];
        o.u = v[kTrajU];
        o.accept = (int)v[kTrajAccept];
        o.cg_iterations = (int)v[kTrajIters];
        o.cg_solves = (int)v[kTrajSolves];
        o.reliable_updates = (int)v[kTrajRU];
        o.max_true_residual = v[kTrajMaxRes];
        o.fp64_iterations = (int)v[kTrajFp64Iters];
        o.status = (int)v[kTrajStatus];
        if (o.cg_solves == 0 && o.status == HMC_OK) o.status = HMC_ERR_TIMEOUT;  // not run
        if (o.status != HMC_OK && first_bad == HMC_OK) first_bad = o.status;
    }
    return first_bad;
}

}  // namespace hmc
