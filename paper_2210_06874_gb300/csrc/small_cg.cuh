// small_cg.cuh -- FP32 iterations of the mixed CG for small lattices on the
// CUDA cores of one thread-block cluster, with E and the iterates resident in
// shared memory.
//
// For V of a few dozen sites the contraction E u of one application is a
// 72 x 72 by 72 x 64 product: far too small to amortise the latency of a
// tensor-core tile (operand build, MMA, TMEM read-back).  Here each CTA of
// the cluster owns a contiguous range of time slices and keeps E^T in FP32
// and the FP32 vectors of its slices in shared memory.
//
// Operator (exponential form): (M u)_t = u_t - s_t E D_{t-1} u_{t-1},
// (M^dag u)_t = u_t - s_{t+1} D_t^* E u_{t+1}, s_0 = -1, D_t = diag e^{i phi_t}.
//
// Each CTA contracts E with the sources of its own slices only: the M^dag
// sources are r_j, the M sources e^{i phi_j} q_j.  The result of the source
// slice whose target belongs to the neighbouring CTA (E r of the first own
// slice, E e^{i phi} q of the last) is sent to that CTA.  The CG direction
// step needs E p' with p' = r + beta p; by linearity E p' = E r + beta E p,
// with E p carried per target slice (wp), so the contraction of M^dag
// depends only on r, final before beta is known, and the one of M only on q,
// final before alpha is known.  Each half iteration therefore runs
//   epilogue -> push the partial norm -> contract -> send the boundary
//   column -> wait -> scalar update,
// and the exchange is byte-counted (st.async with mbarrier complete_tx on
// the receiver's barrier, which its owner arms with the expected byte count):
// the partial norms and the boundary column complete the receiver's phase,
// with no release fence on the sending side.
#pragma once

#include "tc_tile.cuh"

namespace hmc {
namespace tc {

constexpr int kSmallMaxSlices = 16;    // time slices per CTA
constexpr int kSmallMaxCluster = 16;   // CTAs per cluster (above 8: non-portable size)

// Shared-memory layout (byte offsets into the operand area; every CTA of the
// cluster uses the same offsets, so a peer's buffer is at the same offset).
struct SmallLayout {
    int V, Vr, S, SP, KS;   // Vr: rows padded to 32; S: most slices of any CTA;
                            // SP: slice stride of the operands (2, 4, 8 or 16);
                            // KS: k parts of a contraction
    uint32_t et;            // float  [V][Vr]   E^T (rows >= V zero)
    uint32_t r, p, x, q;    // float2 [S][V]    own slices
    uint32_t wp;            // float2 [S][V]    E p of the source of each own target slice
    uint32_t cis;           // float2 [S][V]    e^{i phi} of the own slices
    uint32_t ud, um;        // float2 [V][SP]   k-major sources of M^dag (r) and M (e^{i phi} q)
    uint32_t bd, bm;        // float2 [V]       boundary columns received from the peers
    uint32_t w;             // float2 [KS][S][Vr] partial products per source slice
    uint32_t total;
};

__host__ __device__ inline uint32_t small_take(uint32_t& o, uint32_t bytes) {
    const uint32_t a = o;
    o += (bytes + 15u) & ~15u;
    return a;
}

__host__ __device__ inline SmallLayout small_layout(int V, int Nt, int C) {
    SmallLayout l;
    l.V = V;
    l.Vr = (V + 31) / 32 * 32;
    l.S = (Nt + C - 1) / C;
    l.SP = l.S <= 2 ? 2 : (l.S <= 4 ? 4 : (l.S <= 8 ? 8 : 16));
    const int G = l.Vr / 32;
    l.KS = G >= 8 ? 1 : 8 / G;
    if (l.KS > V) l.KS = V;
    uint32_t o = 0;
    l.et = small_take(o, (uint32_t)V * l.Vr * 4);
    const uint32_t vb = (uint32_t)l.S * V * 8;
    l.r = small_take(o, vb);
    l.p = small_take(o, vb);
    l.x = small_take(o, vb);
    l.q = small_take(o, vb);
    l.wp = small_take(o, vb);
    l.cis = small_take(o, vb);
    l.ud = small_take(o, (uint32_t)V * l.SP * 8);
    l.um = small_take(o, (uint32_t)V * l.SP * 8);
    l.bd = small_take(o, (uint32_t)V * 8);
    l.bm = small_take(o, (uint32_t)V * 8);
    l.w = small_take(o, (uint32_t)l.KS * l.S * l.Vr * 8);
    l.total = o;
    return l;
}

// The cluster layout fits: C in [1, 16], every CTA owns 1..16 slices, and
// the buffers fit the operand area.
__host__ __device__ inline bool small_feasible(int V, int Nt, int C) {
    if (C < 1 || C > kSmallMaxCluster || Nt < C) return false;
    if ((Nt + C - 1) / C > kSmallMaxSlices) return false;
    return small_layout(V, Nt, C).total <= kOperandBytes;
}

// Store an FP32 pair at the same offset in the shared memory of cluster CTA
// `rank` (a plain store when the cluster is this CTA alone).
__device__ __forceinline__ void st_peer(float2* p, uint32_t rank, int C, float2 v) {
    if (C == 1) {
        *p = v;
        return;
    }
    uint32_t a = cta_smem_u32(p), ra;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(a), "r"(rank));
    asm volatile("st.shared::cluster.v2.f32 [%0], {%1, %2};" ::"r"(ra), "f"(v.x), "f"(v.y)
                 : "memory");
}

// Walk elements e = tid, tid + nthr, ... of a slice-major [S][V] block with
// their (slice j, site k), advancing (j, k) without a division per element.
struct SliceWalk {
    int j, k, dj, dk, V;
    __device__ __forceinline__ explicit SliceWalk(int V_) : V(V_) {
        dj = (int)blockDim.x / V;
        dk = (int)blockDim.x - dj * V;
        j = (int)threadIdx.x / V;
        k = (int)threadIdx.x - j * V;
    }
    __device__ __forceinline__ void next() {
        j += dj;
        k += dk;
        if (k >= V) {
            k -= V;
            ++j;
        }
    }
};

// Per-CTA view of the cluster solver.
struct SmallCg {
    SmallLayout l;
    uint8_t* base;
    int rank, C, Nt;
    int t_lo, S;        // own slices t_lo .. t_lo+S-1
    int prev, next;     // cluster ranks owning slices t_lo-1 and t_lo+S (mod Nt)
    __device__ __forceinline__ float2* v(uint32_t off) const {
        return reinterpret_cast<float2*>(base + off);
    }
    __device__ __forceinline__ float* et() const { return reinterpret_cast<float*>(base + l.et); }
};

__device__ __forceinline__ int small_t_lo(int c, int Nt, int C) { return (c * Nt) / C; }

__device__ inline void small_init_view(SmallCg& sc, uint8_t* base, int rank, int C, int V,
                                       int Nt) {
    sc.l = small_layout(V, Nt, C);
    sc.base = base;
    sc.rank = rank;
    sc.C = C;
    sc.Nt = Nt;
    sc.t_lo = small_t_lo(rank, Nt, C);
    sc.S = small_t_lo(rank + 1, Nt, C) - sc.t_lo;
    sc.prev = rank == 0 ? C - 1 : rank - 1;
    sc.next = rank == C - 1 ? 0 : rank + 1;
}

// Per-solve set-up of this CTA: E^T in FP32, the phases of its slices,
// r = chi (FP32), p = x = E p = 0, zero operands (their padding columns
// stay zero).  Returns this thread's FP64 partial |r|^2.
__device__ inline double small_setup(SmallCg& sc, const ChainView& c, const double2* chi) {
    const SmallLayout& l = sc.l;
    const int V = l.V, nthr = blockDim.x;
    float* Et = sc.et();
    for (int e = threadIdx.x; e < V * l.Vr; e += nthr) {
        const int k = e / l.Vr, i = e - k * l.Vr;
        Et[e] = i < V ? (float)c.E[(size_t)i * V + k] : 0.f;
    }
    float2* cis = sc.v(l.cis);
    const size_t g0 = (size_t)sc.t_lo * V;
    const int n = sc.S * V;
    for (int e = threadIdx.x; e < n; e += nthr) cis[e] = c.cis_f[g0 + e];
    float2 *r = sc.v(l.r), *p = sc.v(l.p), *x = sc.v(l.x), *wp = sc.v(l.wp);
    const float2 z = make_float2(0.f, 0.f);
    double acc = 0.0;
    for (int e = threadIdx.x; e < n; e += nthr) {
        const double2 ch = chi[g0 + e];
        const float2 rv = make_float2((float)ch.x, (float)ch.y);
        r[e] = rv;
        p[e] = z;
        x[e] = z;
        wp[e] = z;
        acc += (double)rv.x * rv.x + (double)rv.y * rv.y;
    }
    float2 *ud = sc.v(l.ud), *um = sc.v(l.um);
    for (int e = threadIdx.x; e < V * l.SP; e += nthr) {
        ud[e] = z;
        um[e] = z;
    }
    return acc;
}

// r = FP32(r64) on this CTA's slices (after a reliable update).
__device__ inline void small_refresh_r(SmallCg& sc, const double2* r64) {
    float2* r = sc.v(sc.l.r);
    const size_t g0 = (size_t)sc.t_lo * sc.l.V;
    for (int e = threadIdx.x; e < sc.S * sc.l.V; e += blockDim.x) {
        const double2 d = r64[g0 + e];
        r[e] = make_float2((float)d.x, (float)d.y);
    }
}

// x64 += x (this CTA's slices), x = 0.
__device__ inline void small_fold_x(SmallCg& sc, double2* x64) {
    float2* x = sc.v(sc.l.x);
    const size_t g0 = (size_t)sc.t_lo * sc.l.V;
    for (int e = threadIdx.x; e < sc.S * sc.l.V; e += blockDim.x) {
        const float2 d = x[e];
        double2 xv = x64[g0 + e];
        xv.x += (double)d.x;
        xv.y += (double)d.y;
        x64[g0 + e] = xv;
        x[e] = make_float2(0.f, 0.f);
    }
}

// ---------------------------------------------------------------- exchange
// Push an FP32 pair into the buffer at the same offset of cluster CTA
// `rank`, byte-counted (8 bytes) on that CTA's barrier of phase kk.
__device__ __forceinline__ void tx_push_pair(const ClusterSync* cs, const float2* p,
                                             uint32_t rank, unsigned kk, float2 v) {
    uint32_t ra, rb;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;"
                 : "=r"(ra)
                 : "r"(cta_smem_u32(p)), "r"(rank));
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;"
                 : "=r"(rb)
                 : "r"(cta_smem_u32(&cs->bar_tx[kk & 1u])), "r"(rank));
    asm volatile(
        "st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.f32 [%0], {%1, %2}, [%3];" ::"r"(
            ra),
        "f"(v.x), "f"(v.y), "r"(rb)
        : "memory");
}

// Warp 0: the CTA's FP32 sum `a` into every member's slot of phase kk,
// byte-counted (4 bytes) on the member's barrier.
__device__ __forceinline__ void tx_push_partial(const Team& tm, unsigned kk, float a) {
    const ClusterSync* cs = tm.cs;
    const int lane = threadIdx.x & 31;
    if (lane < tm.size) {
        uint32_t ra, rb;
        asm volatile("mapa.shared::cluster.u32 %0, %1, %2;"
                     : "=r"(ra)
                     : "r"(cta_smem_u32(&cs->part_tx[kk & 1u][tm.rank])), "r"(lane));
        asm volatile("mapa.shared::cluster.u32 %0, %1, %2;"
                     : "=r"(rb)
                     : "r"(cta_smem_u32(&cs->bar_tx[kk & 1u])), "r"(lane));
        asm volatile(
            "st.async.shared::cluster.mbarrier::complete_tx::bytes.f32 [%0], %1, [%2];" ::"r"(ra),
            "f"(a), "r"(rb)
            : "memory");
    }
}

// Lane 0: arm phase kk (one arrival, `bytes` expected) and wait for it,
// bounded.  False on timeout or team failure.
__device__ inline bool tx_wait(const Team& tm, unsigned kk, uint32_t bytes) {
    ClusterSync* cs = tm.cs;
    const uint32_t bar = cta_smem_u32(&cs->bar_tx[kk & 1u]);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
    const uint32_t phase = (kk >> 1) & 1u;
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

// Split-phase FP32 sum of one value per thread over the cluster (or the one
// CTA).  begin: fixed-order CTA sum (warp shuffles, then a shuffle tree over
// the warp sums) pushed to every member by warp 0.  end: waits for phase kk
// (the partials plus the boundary column from the neighbour) and returns the
// members' sums added in rank order, on every thread.
struct SmallSum {
    float w[32];
    float single;
    float tot;
    int ok;
};

__device__ inline void small_sum_begin(const Team& tm, SmallSum& ss, unsigned kk, float x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    if (lane == 0) ss.w[warp] = x;
    __syncthreads();
    if (warp == 0) {
        float a = lane < nw ? ss.w[lane] : 0.f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
        a = __shfl_sync(0xffffffffu, a, 0);
        if (tm.size == 1) {
            if (lane == 0) ss.single = a;
        } else {
            tx_push_partial(tm, kk, a);
        }
    }
}

__device__ inline bool small_sum_end(const Team& tm, SmallSum& ss, unsigned kk, uint32_t bytes,
                                     float& out) {
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        if (tm.size == 1) {
            if (lane == 0) {
                ss.tot = ss.single;
                ss.ok = 1;
            }
        } else {
            bool ok = true;
            if (lane == 0) ok = tx_wait(tm, kk, bytes);
            __syncwarp();
            float b = lane < tm.size ? tm.cs->part_tx[kk & 1u][lane] : 0.f;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) b += __shfl_down_sync(0xffffffffu, b, o);
            if (lane == 0) {
                ss.tot = b;
                ss.ok = ok ? 1 : 0;
            }
        }
    }
    __syncthreads();
    out = ss.tot;
    return ss.ok != 0;
}

// ---------------------------------------------------------------- compute
// The sources of the M^dag contraction, ud[k][j] = r_j[k] (all own slices);
// used at segment start.
__device__ inline void small_load_ud(SmallCg& sc) {
    const SmallLayout& l = sc.l;
    const int V = l.V, n = sc.S * V;
    const float2* r = sc.v(l.r);
    float2* ud = sc.v(l.ud);
    SliceWalk it(V);
    for (int e = threadIdx.x; e < n; e += blockDim.x, it.next()) ud[it.k * l.SP + it.j] = r[e];
}

// W[h][j][i] = sum over k in part h of E[i][k] U[k][j] for all SP columns of
// a k-major operand (padding columns give zero).  Warp w takes (row group,
// k part) items, lane = row; the operand row of one k is a broadcast read;
// the loads of UNR consecutive k are issued before their products.
template <int SP>
__device__ inline void small_matvec(const SmallCg& sc, const float2* U) {
    constexpr int H = SP / 2;                      // float4 per operand row
    constexpr int UNR = SP <= 4 ? 4 : (SP <= 8 ? 2 : 1);
    const SmallLayout& l = sc.l;
    const float* Et = sc.et();
    const float4* U4 = reinterpret_cast<const float4*>(U);
    float2* W = sc.v(l.w);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const int G = l.Vr / 32, items = G * l.KS;
    // with fewer items than warps the last warps take them: warp 0 is then
    // still sending the partial norm of the epilogue before (small_sum_begin)
    const int w0 = items < nw ? nw - items : 0;
    for (int item = warp - w0; warp >= w0 && item < items; item += nw - w0) {
        const int g = item % G, h = item / G;
        const int i = g * 32 + lane;
        const int k0 = (h * l.V) / l.KS, k1 = ((h + 1) * l.V) / l.KS;
        float ar[SP], ai[SP];
#pragma unroll
        for (int j = 0; j < SP; ++j) {
            ar[j] = 0.f;
            ai[j] = 0.f;
        }
        int k = k0;
        for (; k + UNR <= k1; k += UNR) {
            float e[UNR];
            float4 u[UNR][H];
#pragma unroll
            for (int q = 0; q < UNR; ++q) {
                e[q] = Et[(k + q) * l.Vr + i];
#pragma unroll
                for (int jj = 0; jj < H; ++jj) u[q][jj] = U4[(size_t)(k + q) * H + jj];
            }
#pragma unroll
            for (int q = 0; q < UNR; ++q)
#pragma unroll
                for (int jj = 0; jj < H; ++jj) {
                    ar[2 * jj] = fmaf(e[q], u[q][jj].x, ar[2 * jj]);
                    ai[2 * jj] = fmaf(e[q], u[q][jj].y, ai[2 * jj]);
                    ar[2 * jj + 1] = fmaf(e[q], u[q][jj].z, ar[2 * jj + 1]);
                    ai[2 * jj + 1] = fmaf(e[q], u[q][jj].w, ai[2 * jj + 1]);
                }
        }
        for (; k < k1; ++k) {
            const float e = Et[k * l.Vr + i];
#pragma unroll
            for (int jj = 0; jj < H; ++jj) {
                const float4 u = U4[(size_t)k * H + jj];
                ar[2 * jj] = fmaf(e, u.x, ar[2 * jj]);
                ai[2 * jj] = fmaf(e, u.y, ai[2 * jj]);
                ar[2 * jj + 1] = fmaf(e, u.z, ar[2 * jj + 1]);
                ai[2 * jj + 1] = fmaf(e, u.w, ai[2 * jj + 1]);
            }
        }
#pragma unroll
        for (int j = 0; j < SP; ++j)
            if (j < sc.S) W[((size_t)h * l.S + j) * l.Vr + i] = make_float2(ar[j], ai[j]);
    }
}

__device__ inline void small_matvec_any(const SmallCg& sc, const float2* U) {
    switch (sc.l.SP) {
        case 2: small_matvec<2>(sc, U); break;
        case 4: small_matvec<4>(sc, U); break;
        case 8: small_matvec<8>(sc, U); break;
        default: small_matvec<16>(sc, U); break;
    }
}

// (E u_src)_i of own source slice j, summed over the k parts in order.
__device__ __forceinline__ float2 small_w(const SmallCg& sc, int j, int i) {
    const float2* W = sc.v(sc.l.w);
    float2 s = W[(size_t)j * sc.l.Vr + i];
    for (int h = 1; h < sc.l.KS; ++h) {
        const float2 t = W[((size_t)h * sc.l.S + j) * sc.l.Vr + i];
        s.x += t.x;
        s.y += t.y;
    }
    return s;
}

// The column of own source slice j whose target is the peer's: into the
// peer's buffer `dst` (byte-counted on phase kk), or into this CTA's own
// buffer when the cluster is this CTA alone.
__device__ inline void small_send_boundary(const SmallCg& sc, const ClusterSync* cs, unsigned kk,
                                           int j, uint32_t dst, uint32_t peer) {
    float2* d = sc.v(dst);
    for (int i = threadIdx.x; i < sc.l.V; i += blockDim.x) {
        const float2 w = small_w(sc, j, i);
        if (sc.C == 1) d[i] = w;
        else tx_push_pair(cs, d + i, peer, kk, w);
    }
}

// Segment start: E r of the first own slice to the previous CTA with plain
// remote stores (a cluster barrier follows).
__device__ inline void small_send_boundary_plain(const SmallCg& sc) {
    float2* d = sc.v(sc.l.bd);
    for (int i = threadIdx.x; i < sc.l.V; i += blockDim.x)
        st_peer(d + i, sc.prev, sc.C, small_w(sc, 0, i));
}

// Direction step, W = E r of the own sources: the target of slice j takes
// column j+1 (the next CTA's boundary column bd for the last slice):
// wp <- W + beta wp (= E p'), p <- r + beta p, q = M^dag p = p - s_{t+1}
// e^{-i phi_t} wp; the M sources um[k][j] <- e^{i phi_j} q_j.  Returns this
// thread's FP32 partial |q|^2.
__device__ inline float small_dag_epilogue(SmallCg& sc, float beta) {
    const SmallLayout& l = sc.l;
    const int V = l.V, n = sc.S * V;
    const float2 *r = sc.v(l.r), *cis = sc.v(l.cis), *bd = sc.v(l.bd);
    float2 *p = sc.v(l.p), *wp = sc.v(l.wp), *q = sc.v(l.q), *um = sc.v(l.um);
    float acc = 0.f;
    SliceWalk it(V);
    for (int e = threadIdx.x; e < n; e += blockDim.x, it.next()) {
        const int j = it.j, i = it.k;
        const float2 wr = j + 1 < sc.S ? small_w(sc, j + 1, i) : bd[i];
        float2 w = wp[e];
        w.x = fmaf(beta, w.x, wr.x);
        w.y = fmaf(beta, w.y, wr.y);
        wp[e] = w;
        const float2 rv = r[e];
        float2 pv = p[e];
        pv.x = fmaf(beta, pv.x, rv.x);
        pv.y = fmaf(beta, pv.y, rv.y);
        p[e] = pv;
        const float2 ph = cis[e];
        const float sg = (sc.t_lo + j == sc.Nt - 1) ? -1.f : 1.f;
        const float cr = ph.x * w.x + ph.y * w.y, ci = ph.x * w.y - ph.y * w.x;   // conj(ph) w
        const float2 qv = make_float2(pv.x - sg * cr, pv.y - sg * ci);
        q[e] = qv;
        acc = fmaf(qv.x, qv.x, fmaf(qv.y, qv.y, acc));
        um[i * l.SP + j] = make_float2(ph.x * qv.x - ph.y * qv.y, ph.x * qv.y + ph.y * qv.x);
    }
    return acc;
}

// Update step, W = E e^{i phi} q of the own sources: the target of slice j
// takes column j-1 (the previous CTA's boundary column bm for the first
// slice): Ap = q - s_t W, x += alpha p, r -= alpha Ap; the M^dag sources
// ud[k][j] <- r_j.  Returns this thread's FP32 partial |r|^2.
__device__ inline float small_m_epilogue(SmallCg& sc, float alpha) {
    const SmallLayout& l = sc.l;
    const int V = l.V, n = sc.S * V;
    const float2 *q = sc.v(l.q), *p = sc.v(l.p), *bm = sc.v(l.bm);
    float2 *x = sc.v(l.x), *r = sc.v(l.r), *ud = sc.v(l.ud);
    float acc = 0.f;
    SliceWalk it(V);
    for (int e = threadIdx.x; e < n; e += blockDim.x, it.next()) {
        const int j = it.j, i = it.k;
        const float2 w = j > 0 ? small_w(sc, j - 1, i) : bm[i];
        const float sg = (sc.t_lo + j == 0) ? -1.f : 1.f;
        const float2 qv = q[e], pv = p[e];
        const float2 ap = make_float2(qv.x - sg * w.x, qv.y - sg * w.y);
        float2 xv = x[e], rv = r[e];
        xv.x = fmaf(alpha, pv.x, xv.x);
        xv.y = fmaf(alpha, pv.y, xv.y);
        rv.x = fmaf(-alpha, ap.x, rv.x);
        rv.y = fmaf(-alpha, ap.y, rv.y);
        x[e] = xv;
        r[e] = rv;
        acc = fmaf(rv.x, rv.x, fmaf(rv.y, rv.y, acc));
        ud[i * l.SP + j] = rv;
    }
    return acc;
}

}  // namespace tc
}  // namespace hmc
