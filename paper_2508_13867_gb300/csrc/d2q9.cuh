// D2Q9 BGK building blocks for the device (arXiv 2508.13867, Sec. 3).
//
// Velocity set and weights: the D2Q9 set and Eq. weightsDdQ9 (4/9, 1/9, 1/36) in the order
// c = (0,0),(1,0),(0,1),(-1,0),(0,-1),(1,1),(-1,1),(-1,-1),(1,-1), with c_s^2 = 1/3.
// Populations are stored shifted, g_i = f_i - w_i, so that low-precision storage spends
// its mantissa on the deviation from rest instead of on the constant w_i.  The BGK update
// (Eq. bgkCollision with Eq. equilibrium) in shifted form reads
//   drho = sum g_i,  j = sum c_i g_i,  rho = 1 + drho,  u = j / rho,
//   g_i^eq = w_i (drho + rho (3 c_i.u + 4.5 (c_i.u)^2 - 1.5 u.u)),
//   g_i*   = g_i + omega (g_i^eq - g_i),
// which is the same arithmetic as f* = f - (f - f^eq)/tau with f = g + w.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cstdint>

namespace uqlb {

__host__ __device__ constexpr int cx(int i) {
    return i == 1 || i == 5 || i == 8 ? 1 : (i == 3 || i == 6 || i == 7 ? -1 : 0);
}
__host__ __device__ constexpr int cy(int i) {
    return i == 2 || i == 5 || i == 6 ? 1 : (i == 4 || i == 7 || i == 8 ? -1 : 0);
}
__host__ __device__ constexpr int opp(int i) {
    return i == 0 ? 0 : (i <= 4 ? ((i + 1) % 4) + 1 : ((i - 5 + 2) % 4) + 5);
}
template <typename C>
__host__ __device__ constexpr C wgt(int i) {
    return i == 0 ? C(4) / C(9) : (i <= 4 ? C(1) / C(9) : C(1) / C(36));
}

static_assert(opp(1) == 3 && opp(2) == 4 && opp(3) == 1 && opp(4) == 2, "opp straight");
static_assert(opp(5) == 7 && opp(6) == 8 && opp(7) == 5 && opp(8) == 6, "opp diagonal");
static_assert(cx(6) == -1 && cy(6) == 1 && cx(8) == 1 && cy(8) == -1, "diagonal order");

// Storage formats of the shifted populations and the arithmetic type used with each.
template <typename S>
struct Storage;
template <>
struct Storage<double> {
    using C = double;
    static __device__ __forceinline__ double load(const double* p) { return *p; }
    static __device__ __forceinline__ void store(double* p, double v) { *p = v; }
};
template <>
struct Storage<float> {
    using C = float;
    static __device__ __forceinline__ float load(const float* p) { return *p; }
    static __device__ __forceinline__ void store(float* p, float v) { *p = v; }
};
template <>
struct Storage<__half> {
    using C = float;
    static __device__ __forceinline__ float load(const __half* p) { return __half2float(*p); }
    static __device__ __forceinline__ void store(__half* p, float v) { *p = __float2half_rn(v); }
};
template <>
struct Storage<__nv_bfloat16> {
    using C = float;
    static __device__ __forceinline__ float load(const __nv_bfloat16* p) {
        return __bfloat162float(*p);
    }
    static __device__ __forceinline__ void store(__nv_bfloat16* p, float v) {
        *p = __float2bfloat16_rn(v);
    }
};

// Moments of shifted populations: drho, u, v (u = j / rho).
template <typename C>
__device__ __forceinline__ void moments(const C g[9], C& drho, C& ux, C& uy) {
    drho = ((g[0] + g[1]) + (g[2] + g[3])) + ((g[4] + g[5]) + (g[6] + g[7])) + g[8];
    const C jx = (g[1] - g[3]) + (g[5] - g[6]) + (g[8] - g[7]);
    const C jy = (g[2] - g[4]) + (g[5] - g[7]) + (g[6] - g[8]);
    const C inv_rho = C(1) / (C(1) + drho);
    ux = jx * inv_rho;
    uy = jy * inv_rho;
}

// BGK relaxation of shifted populations towards the shifted equilibrium, in place.
template <typename C>
__device__ __forceinline__ void bgk(C g[9], C omega, C drho, C ux, C uy) {
    const C rho = C(1) + drho;
    const C usq15 = C(1.5) * (ux * ux + uy * uy);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const C cu = C(cx(i)) * ux + C(cy(i)) * uy;
        const C geq = wgt<C>(i) * (drho + rho * (C(3) * cu + C(4.5) * cu * cu - usq15));
        g[i] = g[i] + omega * (geq - g[i]);
    }
}

// Obstacle bitmask lookup: bit (x & 31) of word y * words + (x >> 5).
__device__ __forceinline__ bool mask_solid(const uint32_t* m, int words, int x, int y) {
    return (__ldg(m + (int64_t)y * words + (x >> 5)) >> (x & 31)) & 1u;
}

}  // namespace uqlb
