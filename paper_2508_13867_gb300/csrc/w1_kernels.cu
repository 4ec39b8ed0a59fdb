// 1-Wasserstein distance between the speed distributions of two ensembles of velocity fields
// (arXiv 2508.13867, Sec. 8.3: W1 of the numerical statistical solutions of |u|).
//
// For two empirical distributions on the real line, W1 is the integral of |F_a(x) - F_b(x)|.
// Both sets of speeds are counted into the same `bins` equal bins over [0, vmax]; the integral
// over the binned CDFs is exact for the binned values, which differ from the true ones by less
// than one bin width h, so |W1_binned - W1| < h.  Three kernels: the largest speed, the two
// histograms (global atomics; the counts do not depend on their order), and one block that
// scans the bins in a fixed order and sums |F_a - F_b| h in FP64.  Non-finite speeds (samples
// that became unstable) are left out of both distributions and counted.
#include <cmath>

#include "uqlb_internal.h"

namespace uqlb {

namespace {

template <typename M>
__device__ __forceinline__ double speed(const M* m, int64_t ld, int64_t nodes, int64_t idx) {
    const int64_t s = idx / nodes, k = idx - s * nodes;
    const double u = (double)m[s * ld + k], v = (double)m[s * ld + nodes + k];
    return sqrt(u * u + v * v);
}

template <typename M>
__global__ void max_speed_kernel(const M* m, int64_t S, int64_t nodes, int64_t ld, unsigned long long* vmax_bits) {
    double best = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < S * nodes; i += (int64_t)gridDim.x * blockDim.x) {
        const double v = speed(m, ld, nodes, i);
        if (isfinite(v)) best = fmax(best, v);
    }
    for (int o = 16; o > 0; o >>= 1) best = fmax(best, __shfl_xor_sync(0xffffffffu, best, o));
    // non-negative doubles order like their bit patterns
    if ((threadIdx.x & 31) == 0) atomicMax(vmax_bits, (unsigned long long)__double_as_longlong(best));
}

// Non-finite speeds (an unstable sample) are not binned; they are counted in *nonfinite.
template <typename M>
__global__ void speed_hist_kernel(const M* m, int64_t S, int64_t nodes, int64_t ld, const unsigned long long* vmax_bits,
                                  int bins, unsigned int* counts, unsigned long long* nonfinite) {
    const double vmax = __longlong_as_double((long long)*vmax_bits);
    const double scale = vmax > 0.0 ? bins / vmax : 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < S * nodes; i += (int64_t)gridDim.x * blockDim.x) {
        const double v = speed(m, ld, nodes, i);
        if (!isfinite(v)) {
            atomicAdd(nonfinite, 1ull);
            continue;
        }
        int b = (int)(v * scale);
        b = b < 0 ? 0 : (b >= bins ? bins - 1 : b);
        atomicAdd(counts + b, 1u);
    }
}

constexpr int kScanThreads = 1024;

__global__ void __launch_bounds__(kScanThreads) w1_scan_kernel(const unsigned int* ca, const unsigned int* cb, int bins,
                                                                double na_all, double nb_all,
                                                                const unsigned long long* vmax_bits,
                                                                const unsigned long long* nonfinite, double* out) {
    const double na = na_all - (double)nonfinite[0], nb = nb_all - (double)nonfinite[1];
    __shared__ long long sa[kScanThreads], sb[kScanThreads];
    __shared__ double sred[kScanThreads / 32];
    const int t = threadIdx.x;
    const int per = (bins + kScanThreads - 1) / kScanThreads;
    const int lo = t * per, hi = min(bins, lo + per);
    long long ta = 0, tb = 0;
    for (int b = lo; b < hi; ++b) {
        ta += ca[b];
        tb += cb[b];
    }
    sa[t] = ta;
    sb[t] = tb;
    __syncthreads();
    // inclusive prefix sums of the chunk totals (Hillis-Steele, fixed order)
    for (int o = 1; o < kScanThreads; o <<= 1) {
        const long long va = t >= o ? sa[t - o] : 0, vb = t >= o ? sb[t - o] : 0;
        __syncthreads();
        sa[t] += va;
        sb[t] += vb;
        __syncthreads();
    }
    long long ra = sa[t] - ta, rb = sb[t] - tb;  // counts before this chunk
    const double h = __longlong_as_double((long long)*vmax_bits) / bins;
    double acc = 0.0;
    for (int b = lo; b < hi; ++b) {
        ra += ca[b];
        rb += cb[b];
        acc += fabs((double)ra / na - (double)rb / nb);
    }
    acc *= h;
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((t & 31) == 0) sred[t >> 5] = acc;
    __syncthreads();
    if (t == 0) {
        double s = 0.0;
        for (int w = 0; w < kScanThreads / 32; ++w) s += sred[w];
        out[0] = (na > 0.0 && nb > 0.0) ? s : NAN;
        out[1] = h;
        out[2] = (double)nonfinite[0];
        out[3] = (double)nonfinite[1];
    }
}

template <typename M>
cudaError_t launch_max(const M* m, int64_t S, int64_t nodes, int64_t ld, unsigned long long* vmax, cudaStream_t s) {
    max_speed_kernel<M><<<1216, 256, 0, s>>>(m, S, nodes, ld, vmax);
    return cudaGetLastError();
}

template <typename M>
cudaError_t launch_hist(const M* m, int64_t S, int64_t nodes, int64_t ld, const unsigned long long* vmax, int bins,
                        unsigned int* counts, unsigned long long* nonfinite, cudaStream_t s) {
    speed_hist_kernel<M><<<1216, 256, 0, s>>>(m, S, nodes, ld, vmax, bins, counts, nonfinite);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_w1_speed(const void* a, int dta, int64_t sa, int64_t na, int64_t lda, const void* b, int dtb,
                            int64_t sb, int64_t nb, int64_t ldb, int bins, void* ws, double* out_dev, cudaStream_t s) {
    auto* vmax = static_cast<unsigned long long*>(ws);
    auto* nonfinite = vmax + 1;  // two counters, one per set
    auto* ca = reinterpret_cast<unsigned int*>(static_cast<char*>(ws) + 256);
    unsigned int* cb = ca + bins;
    cudaError_t e;
    if ((e = cudaMemsetAsync(ws, 0, 256 + (size_t)2 * bins * sizeof(unsigned int), s))) return e;
    e = dta == UQLB_F64 ? launch_max(static_cast<const double*>(a), sa, na, lda, vmax, s)
                        : launch_max(static_cast<const float*>(a), sa, na, lda, vmax, s);
    if (e) return e;
    e = dtb == UQLB_F64 ? launch_max(static_cast<const double*>(b), sb, nb, ldb, vmax, s)
                        : launch_max(static_cast<const float*>(b), sb, nb, ldb, vmax, s);
    if (e) return e;
    e = dta == UQLB_F64 ? launch_hist(static_cast<const double*>(a), sa, na, lda, vmax, bins, ca, nonfinite, s)
                        : launch_hist(static_cast<const float*>(a), sa, na, lda, vmax, bins, ca, nonfinite, s);
    if (e) return e;
    e = dtb == UQLB_F64 ? launch_hist(static_cast<const double*>(b), sb, nb, ldb, vmax, bins, cb, nonfinite + 1, s)
                        : launch_hist(static_cast<const float*>(b), sb, nb, ldb, vmax, bins, cb, nonfinite + 1, s);
    if (e) return e;
    w1_scan_kernel<<<1, kScanThreads, 0, s>>>(ca, cb, bins, (double)(sa * na), (double)(sb * nb), vmax, nonfinite,
                                              out_dev);
    return cudaGetLastError();
}

}  // namespace uqlb
