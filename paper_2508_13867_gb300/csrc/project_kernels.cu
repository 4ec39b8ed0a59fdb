// gPC projection and ensemble statistics (arXiv 2508.13867, Sec. 4 and Algorithm 1).
//
//   coefficients (Eq. coef_discrete, gamma_k = 1):  C[k, f] = sum_s W[k, s] M[s, f],
//                                                     W[k, s] = a_s Phi_k(xi_s)
//   gPC mean / variance (Eq. gpc_mean, Eq. gpc_std):  mean = C[0, f], var = sum_{k>=1} C[k, f]^2
//   Monte Carlo (Eq. meanMCS, Eq. varMCS):           two passes over the samples
// All accumulation is FP64; M may be FP32 (the ensemble's field output) or FP64.
// The contraction is [K x S] x [S x F] with K <= a few hundred and F up to ~10^6: each thread
// owns two fields and KB coefficients, W tiles are staged in shared memory and broadcast.
#include <cmath>
#include <cstdio>
#include <mutex>

#include "uqlb_internal.h"

namespace uqlb {

namespace {

constexpr int kProjThreads = 128;
constexpr int kKB = 16;   // coefficients per block (blockIdx.y chunk)
constexpr int kSB = 128;  // samples per shared-memory stage
constexpr int kFPT = 2;   // fields per thread

template <typename M>
__global__ void __launch_bounds__(kProjThreads) project_kernel(const double* __restrict__ W, int K, int S,
                                                               const M* __restrict__ m, int64_t F, int64_t ld,
                                                               double* __restrict__ C) {
    __shared__ double sw[kKB][kSB];
    const int k0 = blockIdx.y * kKB;
    const int64_t f0 = ((int64_t)blockIdx.x * kProjThreads) * kFPT + threadIdx.x;
    double acc[kFPT][kKB];
#pragma unroll
    for (int a = 0; a < kFPT; ++a)
#pragma unroll
        for (int k = 0; k < kKB; ++k) acc[a][k] = 0.0;

    for (int s0 = 0; s0 < S; s0 += kSB) {
        const int sn = min(kSB, S - s0);
        for (int q = threadIdx.x; q < kKB * kSB; q += kProjThreads) {
            const int kk = q / kSB, ss = q % kSB;
            sw[kk][ss] = (k0 + kk < K && ss < sn) ? W[(int64_t)(k0 + kk) * S + s0 + ss] : 0.0;
        }
        __syncthreads();
        for (int ss = 0; ss < sn; ++ss) {
            const M* row = m + (int64_t)(s0 + ss) * ld;
            double v[kFPT];
#pragma unroll
            for (int a = 0; a < kFPT; ++a) {
                const int64_t f = f0 + (int64_t)a * kProjThreads;
                v[a] = f < F ? (double)row[f] : 0.0;
            }
#pragma unroll
            for (int k = 0; k < kKB; ++k) {
                const double w = sw[k][ss];
#pragma unroll
                for (int a = 0; a < kFPT; ++a) acc[a][k] = fma(w, v[a], acc[a][k]);
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < kFPT; ++a) {
        const int64_t f = f0 + (int64_t)a * kProjThreads;
        if (f >= F) continue;
#pragma unroll
        for (int k = 0; k < kKB; ++k)
            if (k0 + k < K) C[(int64_t)(k0 + k) * F + f] = acc[a][k];
    }
}

__global__ void gpc_stats_kernel(const double* __restrict__ C, int K, int64_t F, double* mean, double* var) {
    for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < F; f += (int64_t)gridDim.x * blockDim.x) {
        double v = 0.0;
        for (int k = 1; k < K; ++k) {
            const double c = C[(int64_t)k * F + f];
            v = fma(c, c, v);
        }
        if (mean) mean[f] = C[f];
        if (var) var[f] = v;
    }
}

// ddof < 0: var receives the sum of squared deviations itself (M2 of a block, for merging blocks).
template <typename M>
__global__ void mc_stats_kernel(const M* __restrict__ m, int64_t S, int64_t F, int64_t ld, double* mean,
                                double* var, int ddof) {
    for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < F; f += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int64_t q = 0; q < S; ++q) s += (double)m[q * ld + f];
        const double mu = s / (double)S;
        double ss = 0.0;
        for (int64_t q = 0; q < S; ++q) {
            const double d = (double)m[q * ld + f] - mu;
            ss = fma(d, d, ss);
        }
        if (mean) mean[f] = mu;
        if (var) var[f] = ddof < 0 ? ss : ((S - ddof) > 0 ? ss / (double)(S - ddof) : NAN);
    }
}

// Sum factorization of the projection on a tensor Gauss-Legendre grid.  There W[k, s] is a product
// over the input dimensions, W[k, s] = prod_q G[alpha_kq][s_q] with G[a][s] = (w_s / 2) phi_a(x_s) (the
// 1-D probability weight times the orthonormal Legendre polynomial), so C = W M contracts one
// dimension at a time, the last (fastest) first.  One stage maps an input T[(r n + s) J' + j'][f] to
// T[r J + o(a, j')][f] = sum_{s < n} G[a][s] T[(r n + s) J' + j'][f] for every degree a that the
// multi-index set admits after the partial index j' (a prefix a = 0 .. c - 1 of the degrees; o(a, j') =
// -1 beyond it; at the last stage o is the coefficient's row k).  A thread owns one field and one
// group (r, j'): it loads the n inputs once and accumulates the c outputs as independent chains, so
// the FP64 pipe (a small fraction of the FP32 rate on GB300) always has several multiply-adds to
// issue.  FP64 throughout.
constexpr int kSfThreads = 256;

template <typename TI>
__global__ void __launch_bounds__(kSfThreads) sf_stage_kernel(const TI* __restrict__ in, int64_t in_ld,
                                                              double* __restrict__ out, int64_t out_ld,
                                                              int64_t groups, int jprev, int jout, int n, int p1,
                                                              const int* __restrict__ oidx,
                                                              const double* __restrict__ G, int64_t F) {
    __shared__ double sG[kSfMaxDegree + 1][kSfMaxPoints];
    for (int q = threadIdx.x; q < (kSfMaxDegree + 1) * kSfMaxPoints; q += kSfThreads) {
        const int a = q / kSfMaxPoints, c = q % kSfMaxPoints;
        sG[a][c] = a < p1 && c < n ? G[a * n + c] : 0.0;
    }
    __syncthreads();
    const int64_t f = (int64_t)blockIdx.x * kSfThreads + threadIdx.x;
    if (f >= F) return;  // no barrier below
    for (int64_t g = blockIdx.y; g < groups; g += gridDim.y) {
        const int64_t r = g / jprev;
        const int jp = (int)(g - r * jprev);
        int cnt = 0;  // admitted degrees: a prefix of 0 .. p1 - 1
#pragma unroll
        for (int a = 0; a <= kSfMaxDegree; ++a)
            if (a < p1 && __ldg(oidx + jp * p1 + a) >= 0) cnt = a + 1;
        double acc[kSfMaxDegree + 1];
#pragma unroll
        for (int a = 0; a <= kSfMaxDegree; ++a) acc[a] = 0.0;
        const TI* src = in + ((r * n) * jprev + jp) * in_ld + f;
        const int64_t step = (int64_t)jprev * in_ld;
#pragma unroll
        for (int q = 0; q < kSfMaxPoints; ++q) {
            if (q < n) {
                const double x = (double)src[q * step];
#pragma unroll
                for (int a = 0; a <= kSfMaxDegree; ++a)
                    if (a < cnt) acc[a] = fma(sG[a][q], x, acc[a]);
            }
        }
#pragma unroll
        for (int a = 0; a <= kSfMaxDegree; ++a)
            if (a < cnt) out[(r * jout + __ldg(oidx + jp * p1 + a)) * out_ld + f] = acc[a];
    }
}

}  // namespace

cudaError_t launch_sf_stage(const void* in, int in_dtype, int64_t in_ld, double* out, int64_t out_ld, int64_t groups,
                            int jprev, int jout, int n, int p1, const int* oidx, const double* G, int64_t F,
                            cudaStream_t s) {
    if (F <= 0 || groups <= 0) return cudaSuccess;
    if (n < 1 || n > kSfMaxPoints || p1 < 1 || p1 > kSfMaxDegree + 1) return cudaErrorInvalidValue;
    dim3 grid((unsigned)((F + kSfThreads - 1) / kSfThreads), (unsigned)(groups < 65535 ? groups : 65535));
    if (in_dtype == UQLB_F64)
        sf_stage_kernel<double><<<grid, kSfThreads, 0, s>>>(static_cast<const double*>(in), in_ld, out, out_ld, groups,
                                                            jprev, jout, n, p1, oidx, G, F);
    else
        sf_stage_kernel<float><<<grid, kSfThreads, 0, s>>>(static_cast<const float*>(in), in_ld, out, out_ld, groups,
                                                           jprev, jout, n, p1, oidx, G, F);
    return cudaGetLastError();
}

cudaError_t launch_project(const double* W, int K, int S, const void* M, int dtype, int64_t F, int64_t ld,
                           double* C, cudaStream_t s) {
    if (F <= 0 || K <= 0) return cudaSuccess;
    const int64_t per_block = (int64_t)kProjThreads * kFPT;
    dim3 grid((unsigned)((F + per_block - 1) / per_block), (unsigned)((K + kKB - 1) / kKB));
    if (dtype == UQLB_F64)
        project_kernel<double><<<grid, kProjThreads, 0, s>>>(W, K, S, static_cast<const double*>(M), F, ld, C);
    else
        project_kernel<float><<<grid, kProjThreads, 0, s>>>(W, K, S, static_cast<const float*>(M), F, ld, C);
    return cudaGetLastError();
}

cudaError_t launch_gpc_stats(const double* C, int K, int64_t F, double* mean, double* var, cudaStream_t s) {
    if (F <= 0) return cudaSuccess;
    const int64_t blocks = (F + 255) / 256;
    gpc_stats_kernel<<<(unsigned)(blocks < 65535 * 8 ? blocks : 65535 * 8), 256, 0, s>>>(C, K, F, mean, var);
    return cudaGetLastError();
}

cudaError_t launch_mc_stats(const void* M, int dtype, int64_t S, int64_t F, int64_t ld, double* mean,
                            double* var, int ddof, cudaStream_t s) {
    if (F <= 0) return cudaSuccess;
    const int64_t blocks = (F + 255) / 256;
    const unsigned g = (unsigned)(blocks < 65535 * 8 ? blocks : 65535 * 8);
    if (dtype == UQLB_F64)
        mc_stats_kernel<double><<<g, 256, 0, s>>>(static_cast<const double*>(M), S, F, ld, mean, var, ddof);
    else
        mc_stats_kernel<float><<<g, 256, 0, s>>>(static_cast<const float*>(M), S, F, ld, mean, var, ddof);
    return cudaGetLastError();
}

}  // namespace uqlb

// =========================================================================================
// Projection without allocation.
//
// Some callers cannot allocate device memory at the moment they need statistics: code running
// under a memory budget that forbids new allocations, host threads that must not take the
// allocator's locks, or embeddings that hand over only their own input and output buffers.
// uqlb_project needs a small device scratch for the weight matrix W, which it takes from a
// caller workspace.  This variant keeps W in a file-scope device array instead, so the caller
// passes nothing but the fields and the coefficient buffer and nothing is allocated.
// =========================================================================================

namespace {

// Capacity of the shared weight-matrix scratch: K x S <= 131072 doubles (1 MiB).  Every GPU
// that loads the library holds this array until the process exits.
constexpr int64_t kNoAllocWMax = 1 << 17;
static __device__ __align__(256) double g_noalloc_w[kNoAllocWMax];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
double* g_noalloc_ptr[kMaxDevices] = {nullptr};

}  // namespace

extern "C" int uqlb_project_noalloc(uqlb_ctx* ctx, const void* m_dev, int dtype, int64_t n_fields, int64_t m_ld,
                                    double* coeffs_dev, void* stream) {
    using namespace uqlb;
    const double* W = nullptr;
    int K = 0, device = 0;
    int64_t S = 0;
    if (int rc = ctx_projection_view(ctx, &W, &K, &S, &device)) return rc;
    if (!m_dev || !coeffs_dev || n_fields < 0 || m_ld < n_fields)
        return ctx_fail(ctx, UQLB_ERR_ARG, "project_noalloc: bad arguments");
    if (dtype != UQLB_F64 && dtype != UQLB_F32)
        return ctx_fail(ctx, UQLB_ERR_ARG, "project_noalloc: dtype must be F64 or F32");
    if ((int64_t)K * S > kNoAllocWMax) {
        char buf[200];
        snprintf(buf, sizeof buf, "project_noalloc: K x S = %lld exceeds the fixed scratch of %lld weights; use uqlb_project",
                 (long long)K * S, (long long)kNoAllocWMax);
        return ctx_fail(ctx, UQLB_ERR_ARG, buf);
    }
    if (device < 0 || device >= kMaxDevices) return ctx_fail(ctx, UQLB_ERR_ARG, "project_noalloc: device index too large");
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) return ctx_fail(ctx, UQLB_ERR_CUDA, cudaGetErrorString(e));
    double* w_dev = nullptr;
    {
        // First call on this device: resolve the device address of the array (host code cannot
        // use the symbol itself, which only stands in for it on the host).  The address is kept for
        // the life of the process; a device reset would invalidate it (documented in the header).
        std::lock_guard<std::mutex> lock(g_noalloc_mutex);
        if (g_noalloc_ptr[device] == nullptr) {
            void* ptr = nullptr;
            e = cudaGetSymbolAddress(&ptr, g_noalloc_w);
            if (e != cudaSuccess) return ctx_fail(ctx, UQLB_ERR_CUDA, cudaGetErrorString(e));
            g_noalloc_ptr[device] = static_cast<double*>(ptr);
        }
        w_dev = g_noalloc_ptr[device];
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // W overwrites exactly the K x S entries the kernel reads, so nothing needs clearing.
    e = cudaMemcpyAsync(w_dev, W, (size_t)K * S * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return ctx_fail(ctx, UQLB_ERR_CUDA, cudaGetErrorString(e));
    e = launch_project(w_dev, K, (int)S, m_dev, dtype, n_fields, m_ld, coeffs_dev, s);
    if (e != cudaSuccess) return ctx_fail(ctx, UQLB_ERR_CUDA, cudaGetErrorString(e));
    return 0;
}
