// brs.cu -- the mixed-differencing fermion operator printed as Eq. (2.2)
// (Brower-Rebbi-Schaich form) and its adjoint, as an HBM-bound stencil.
//
// With phi the phase angle (delta * phi_paper) and dk = delta * kappa:
//   A site x, slice t:  (M psi) = psi_{x,t+1} - e^{+i phi_{x,t}} psi_{x,t} - dk sum_<y> psi_{y,t}
//   B site x, slice t:  (M psi) = psi_{x,t}   - e^{-i phi_{x,t}} psi_{x,t-1} - dk sum_<y> psi_{y,t}
// antiperiodic in time (psi_{x,Nt} = -psi_{x,0}, psi_{x,-1} = -psi_{x,Nt-1}).
// Adjoint:
//   A:  (M^dag psi) = psi_{x,t-1} - e^{-i phi_{x,t}} psi_{x,t}   - dk sum psi_{y,t}
//   B:  (M^dag psi) = psi_{x,t}   - e^{+i phi_{x,t+1}} psi_{x,t+1} - dk sum psi_{y,t}
// The three neighbours of a site are on the other sublattice of the same
// slice: A(m1,m2) ~ B(m1,m2), B(m1-1,m2), B(m1,m2-1); B(m1,m2) ~ A(m1,m2),
// A(m1+1,m2), A(m1,m2+1) (indices mod L), so a warp of consecutive sites
// reads consecutive neighbours.  Two outputs per thread, one slice per
// grid row: the vector, the phase table and the output each cross HBM once;
// neighbour and time-neighbour re-reads hit L1/L2.
#include <cmath>
#include <cstdint>

#include "common.cuh"

namespace hmc {
namespace brs {

template <typename T>
struct C2;
template <>
struct C2<double> {
    using type = double2;
};
template <>
struct C2<float> {
    using type = float2;
};

template <typename T>
__device__ __forceinline__ typename C2<T>::type cm(typename C2<T>::type a,
                                                   typename C2<T>::type b) {
    return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename T>
__device__ __forceinline__ typename C2<T>::type cmc(typename C2<T>::type a,
                                                    typename C2<T>::type b) {  // conj(a) b
    return {a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x};
}

// cis64[e] = e^{i phi[e]} (FP64), cis32[e] = the same rounded to FP32.
__global__ void k_phases(const double* __restrict__ phi, double2* __restrict__ cis64,
                         float2* __restrict__ cis32, long long N) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < N;
         e += (long long)gridDim.x * blockDim.x) {
        double s, c;
        sincos(phi[e], &s, &c);
        if (cis64) cis64[e] = make_double2(c, s);
        if (cis32) cis32[e] = make_float2((float)c, (float)s);
    }
}

// One output site-slice; blockIdx.y is the slice, so no 64-bit division.
template <typename T, bool DAG>
__device__ __forceinline__ typename C2<T>::type site(int L, int LL, int V, int Nt, int t, int x,
                                                     T dk, const typename C2<T>::type* cis,
                                                     const typename C2<T>::type* in) {
    using T2 = typename C2<T>::type;
    const bool isB = x >= LL;
    const int cidx = isB ? x - LL : x;
    const int m1 = cidx / L, m2 = cidx - m1 * L;
    const T2* row = in + (size_t)t * V;
    int y0, y1, y2;
    if (!isB) {
        y0 = LL + cidx;
        y1 = LL + (m1 == 0 ? L - 1 : m1 - 1) * L + m2;
        y2 = LL + m1 * L + (m2 == 0 ? L - 1 : m2 - 1);
    } else {
        y0 = cidx;
        y1 = (m1 == L - 1 ? 0 : m1 + 1) * L + m2;
        y2 = m1 * L + (m2 == L - 1 ? 0 : m2 + 1);
    }
    const T2 a = row[y0], b = row[y1], c = row[y2];
    const T2 self = row[x];
    const bool up = DAG ? isB : !isB;   // forward time neighbour needed
    int tn;
    T sg = (T)1;
    if (up) {
        tn = t + 1;
        if (tn == Nt) { tn = 0; sg = (T)-1; }
    } else {
        tn = t - 1;
        if (tn < 0) { tn = Nt - 1; sg = (T)-1; }
    }
    T2 nb = in[(size_t)tn * V + x];
    nb.x *= sg;
    nb.y *= sg;
    T2 r;
    if (!DAG) {
        if (!isB) {   // psi_{t+1} - e^{i phi_t} psi_t
            const T2 w = cm<T>(cis[(size_t)t * V + x], self);
            r = {nb.x - w.x, nb.y - w.y};
        } else {      // psi_t - e^{-i phi_t} psi_{t-1}
            const T2 w = cmc<T>(cis[(size_t)t * V + x], nb);
            r = {self.x - w.x, self.y - w.y};
        }
    } else {
        if (!isB) {   // psi_{t-1} - e^{-i phi_t} psi_t
            const T2 w = cmc<T>(cis[(size_t)t * V + x], self);
            r = {nb.x - w.x, nb.y - w.y};
        } else {      // psi_t - e^{i phi_{t+1}} psi_{t+1}  (phase of the wrapped t+1)
            const T2 w = cm<T>(cis[(size_t)tn * V + x], nb);
            r = {self.x - w.x, self.y - w.y};
        }
    }
    return {r.x - dk * (a.x + b.x + c.x), r.y - dk * (a.y + b.y + c.y)};
}

// grid (ceil(V / (2*256)), Nt): each thread writes two consecutive sites.
template <typename T, bool DAG>
__global__ void __launch_bounds__(256) k_apply(int L, int Nt, T dk,
                                               const typename C2<T>::type* __restrict__ cis,
                                               const typename C2<T>::type* __restrict__ in,
                                               typename C2<T>::type* __restrict__ out) {
    const int LL = L * L, V = 2 * LL;
    const int t = blockIdx.y;
    const int x0 = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    if (x0 >= V) return;
    typename C2<T>::type* o = out + (size_t)t * V;
    o[x0] = site<T, DAG>(L, LL, V, Nt, t, x0, dk, cis, in);
    if (x0 + 1 < V) o[x0 + 1] = site<T, DAG>(L, LL, V, Nt, t, x0 + 1, dk, cis, in);
}

// FP32, even L: the two sites x0, x0+1 (x0 even) share a row of the
// lattice (L even) and a sublattice (L*L even), so the vector, the phase
// table, the output, the time neighbour and two of the three spatial
// neighbours of the pair are contiguous 16-byte float4 accesses; only the
// neighbour that wraps in m2 is read per site.
template <bool DAG>
__global__ void __launch_bounds__(256) k_apply_f32_pairs(int L, int Nt, float dk,
                                                         const float4* __restrict__ cis,
                                                         const float4* __restrict__ in,
                                                         float4* __restrict__ out) {
    const int LL = L * L, V = 2 * LL, V2 = LL;   // float4 per slice = V / 2
    const int t = blockIdx.y;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;   // pair index in the slice
    if (p >= V2) return;
    const int x0 = 2 * p;
    const bool isB = x0 >= LL;
    const int cidx = isB ? x0 - LL : x0;
    const int m1 = cidx / L, m2 = cidx - m1 * L;           // m2 even
    const float2* row2 = reinterpret_cast<const float2*>(in) + (size_t)t * V;
    const float4* row4 = in + (size_t)t * V2;
    float4 n0, n1;
    float2 w0, w1;   // the wrapping neighbour of site 0 and site 1
    if (!isB) {
        n0 = row4[(LL + cidx) >> 1];                                   // B(m1, m2)
        n1 = row4[(LL + (m1 == 0 ? L - 1 : m1 - 1) * L + m2) >> 1];      // B(m1-1, m2)
        w0 = row2[LL + m1 * L + (m2 == 0 ? L - 1 : m2 - 1)];             // B(m1, m2-1)
        w1 = row2[LL + m1 * L + m2];                                     // B(m1, m2) for m2+1
    } else {
        n0 = row4[cidx >> 1];                                          // A(m1, m2)
        n1 = row4[((m1 == L - 1 ? 0 : m1 + 1) * L + m2) >> 1];         // A(m1+1, m2)
        w0 = row2[m1 * L + m2 + 1];                                    // A(m1, m2+1)
        w1 = row2[m1 * L + (m2 + 2 == L ? 0 : m2 + 2)];                // A(m1, m2+2)
    }
    const float4 self = row4[p];
    const bool up = DAG ? isB : !isB;
    int tn;
    float sg = 1.f;
    if (up) {
        tn = t + 1;
        if (tn == Nt) { tn = 0; sg = -1.f; }
    } else {
        tn = t - 1;
        if (tn < 0) { tn = Nt - 1; sg = -1.f; }
    }
    float4 nb = in[(size_t)tn * V2 + p];
    nb.x *= sg; nb.y *= sg; nb.z *= sg; nb.w *= sg;
    const float4 ph = cis[(size_t)((DAG && isB) ? tn : t) * V2 + p];
    float2 r0, r1;
    const float2 s0 = make_float2(self.x, self.y), s1 = make_float2(self.z, self.w);
    const float2 b0 = make_float2(nb.x, nb.y), b1 = make_float2(nb.z, nb.w);
    const float2 c0 = make_float2(ph.x, ph.y), c1 = make_float2(ph.z, ph.w);
    if (!DAG) {
        if (!isB) {
            const float2 u0 = cm<float>(c0, s0), u1 = cm<float>(c1, s1);
            r0 = make_float2(b0.x - u0.x, b0.y - u0.y);
            r1 = make_float2(b1.x - u1.x, b1.y - u1.y);
        } else {
            const float2 u0 = cmc<float>(c0, b0), u1 = cmc<float>(c1, b1);
            r0 = make_float2(s0.x - u0.x, s0.y - u0.y);
            r1 = make_float2(s1.x - u1.x, s1.y - u1.y);
        }
    } else {
        if (!isB) {
            const float2 u0 = cmc<float>(c0, s0), u1 = cmc<float>(c1, s1);
            r0 = make_float2(b0.x - u0.x, b0.y - u0.y);
            r1 = make_float2(b1.x - u1.x, b1.y - u1.y);
        } else {
            const float2 u0 = cm<float>(c0, b0), u1 = cm<float>(c1, b1);
            r0 = make_float2(s0.x - u0.x, s0.y - u0.y);
            r1 = make_float2(s1.x - u1.x, s1.y - u1.y);
        }
    }
    const float h0x = n0.x + n1.x + w0.x, h0y = n0.y + n1.y + w0.y;
    const float h1x = n0.z + n1.z + w1.x, h1y = n0.w + n1.w + w1.y;
    out[(size_t)t * V2 + p] =
        make_float4(r0.x - dk * h0x, r0.y - dk * h0y, r1.x - dk * h1x, r1.y - dk * h1y);
}

static int grid_for(long long N, int threads) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    long long g = (N + threads - 1) / threads;
    const long long cap = (long long)(sms > 0 ? sms : 148) * 16;
    return (int)(g < cap ? (g < 1 ? 1 : g) : cap);
}

}  // namespace brs
}  // namespace hmc

extern "C" {

int hmc_brs_phases(int L, int Nt, const double* phi, void* cis64, void* cis32, void* stream) {
    if (L < 1 || Nt < 1 || !phi || (!cis64 && !cis32)) return HMC_ERR_BAD_ARG;
    const long long N = 2LL * L * L * Nt;
    hmc::brs::k_phases<<<hmc::brs::grid_for(N, 256), 256, 0, (cudaStream_t)stream>>>(
        phi, (double2*)cis64, (float2*)cis32, N);
    return cudaGetLastError() == cudaSuccess ? HMC_OK : HMC_ERR_CUDA;
}

int hmc_apply_brs(int L, int Nt, double delta_kappa, const void* cis, const void* in, void* out,
                  int prec, int dagger, void* stream) {
    if (L < 1 || Nt < 1 || !cis || !in || !out || in == out) return HMC_ERR_BAD_ARG;
    if (!std::isfinite(delta_kappa)) return HMC_ERR_BAD_ARG;
    const long long N = 2LL * L * L * Nt;
    if (N >= (1LL << 31) || Nt > 65535) return HMC_ERR_UNSUPPORTED;
    const int V = 2 * L * L;
    const dim3 g((V + 511) / 512, Nt);
    cudaStream_t s = (cudaStream_t)stream;
    using namespace hmc::brs;
    if (prec == HMC_PREC_FP64) {
        if (dagger)
            k_apply<double, true><<<g, 256, 0, s>>>(L, Nt, delta_kappa, (const double2*)cis,
                                                    (const double2*)in, (double2*)out);
        else
            k_apply<double, false><<<g, 256, 0, s>>>(L, Nt, delta_kappa, (const double2*)cis,
                                                     (const double2*)in, (double2*)out);
    } else if (prec == HMC_PREC_MIXED && (L % 2) == 0 &&
               ((reinterpret_cast<uintptr_t>(cis) | reinterpret_cast<uintptr_t>(in) |
                 reinterpret_cast<uintptr_t>(out)) & 15) == 0) {
        const dim3 g2((V / 2 + 255) / 256, Nt);
        if (dagger)
            k_apply_f32_pairs<true><<<g2, 256, 0, s>>>(L, Nt, (float)delta_kappa,
                                                       (const float4*)cis, (const float4*)in,
                                                       (float4*)out);
        else
            k_apply_f32_pairs<false><<<g2, 256, 0, s>>>(L, Nt, (float)delta_kappa,
                                                        (const float4*)cis, (const float4*)in,
                                                        (float4*)out);
    } else if (prec == HMC_PREC_MIXED) {
        if (dagger)
            k_apply<float, true><<<g, 256, 0, s>>>(L, Nt, (float)delta_kappa, (const float2*)cis,
                                                   (const float2*)in, (float2*)out);
        else
            k_apply<float, false><<<g, 256, 0, s>>>(L, Nt, (float)delta_kappa,
                                                    (const float2*)cis, (const float2*)in,
                                                    (float2*)out);
    } else {
        return HMC_ERR_BAD_ARG;
    }
    return cudaGetLastError() == cudaSuccess ? HMC_OK : HMC_ERR_CUDA;
}

}  // extern "C"
