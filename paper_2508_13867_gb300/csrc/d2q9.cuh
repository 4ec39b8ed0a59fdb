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
// rho itself is never rounded: 1/rho - 1 = -drho/(1 + drho) is carried as a small correction
// and the rho-weighted equilibrium terms are written on j = rho u, so reduced-precision
// rounding is relative to drho (~1e-4) and to j, never to 1.
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
// load(p, q, i) / store(p, v, q, i) convert population i (q: the sample's quanta, used by the
// fixed-point format only); store() rounds to nearest even; store_sr() rounds stochastically with
// 16 random bits r: the magnitude is rounded up with probability equal to the discarded fraction,
// so rounding errors have zero mean.  This matters for 16-bit storage on fine lattices, where the
// change of g over one step is far below one unit in the last place and nearest rounding keeps
// discarding it with a consistent sign (stagnation).  at_limit(p) tells whether a stored value sits
// at the end of the format's range (the fixed-point format saturates there).

// Velocity class of population i: 0 rest, 1 axis, 2 diagonal (opposite directions share it).
__host__ __device__ constexpr int qclass(int i) { return i == 0 ? 0 : (i <= 4 ? 1 : 2); }

// Quanta of the 16-bit fixed-point format for one sample: g_i = q * d[qclass(i)] with q a signed
// 16-bit integer, inv = 1 / d.  Formats that need none take NoQuanta.
struct Quanta {
    float d[3];
    float inv[3];
};
struct NoQuanta {};

template <typename S>
struct Storage;
template <>
struct Storage<double> {
    using C = double;
    using Q = NoQuanta;
    static __device__ __forceinline__ double load(const double* p, const Q&, int) { return *p; }
    static __device__ __forceinline__ void store(double* p, double v, const Q&, int) { *p = v; }
    static __device__ __forceinline__ void store_sr(double* p, double v, uint32_t, const Q&, int) { *p = v; }
    static __device__ __forceinline__ bool at_limit(const double*) { return false; }
};
template <>
struct Storage<float> {
    using C = float;
    using Q = NoQuanta;
    static __device__ __forceinline__ float load(const float* p, const Q&, int) { return *p; }
    static __device__ __forceinline__ void store(float* p, float v, const Q&, int) { *p = v; }
    static __device__ __forceinline__ void store_sr(float* p, float v, uint32_t, const Q&, int) { *p = v; }
    static __device__ __forceinline__ bool at_limit(const float*) { return false; }
};
// FP16 holds g scaled by 2^12 (exact): |g| <= ~0.05 then stays far below the FP16 maximum and
// values down to 1.5e-8 stay in the normal range, where the rounding step is relative.
template <>
struct Storage<__half> {
    using C = float;
    using Q = NoQuanta;
    static __device__ __forceinline__ float load(const __half* p, const Q&, int) { return __half2float(*p) * 0x1p-12f; }
    static __device__ __forceinline__ void store(__half* p, float v, const Q&, int) { *p = __float2half_rn(v * 0x1p12f); }
    // 13 random bits below the last FP16 mantissa place of the FP32 pattern, then truncation
    static __device__ __forceinline__ void store_sr(__half* p, float v, uint32_t r, const Q&, int) {
        *p = __float2half_rz(__uint_as_float(__float_as_uint(v * 0x1p12f) + (r & 0x1FFFu)));
    }
    static __device__ __forceinline__ bool at_limit(const __half*) { return false; }
};
template <>
struct Storage<__nv_bfloat16> {
    using C = float;
    using Q = NoQuanta;
    static __device__ __forceinline__ float load(const __nv_bfloat16* p, const Q&, int) { return __bfloat162float(*p); }
    static __device__ __forceinline__ void store(__nv_bfloat16* p, float v, const Q&, int) { *p = __float2bfloat16_rn(v); }
    // 16 random bits added below the BF16 mantissa of the FP32 pattern, then truncation
    static __device__ __forceinline__ void store_sr(__nv_bfloat16* p, float v, uint32_t r, const Q&, int) {
        *p = __ushort_as_bfloat16((unsigned short)((__float_as_uint(v) + (r & 0xFFFFu)) >> 16));
    }
    static __device__ __forceinline__ bool at_limit(const __nv_bfloat16*) { return false; }
};

// 16-bit fixed point: g_i = q d_c, q a signed 16-bit integer, with one quantum d_c per sample and
// velocity class c (rest, axis, diagonal) sized by the host from a bound on |g_i| over the run.
// Every stored value carries the same absolute resolution d_c: the error of the velocity field is
// an absolute error summed over populations, so no bits go to an exponent that |g| never uses
// (FP16 keeps 11 significant bits, BF16 8; here 15 bits span the class's range).  Stores saturate
// at -32768 and 32767; a sample holding a saturated value at its end is reported unstable.
template <>
struct Storage<int16_t> {
    using C = float;
    using Q = Quanta;
    static __device__ __forceinline__ float load(const int16_t* p, const Q& q, int i) {
        return (float)*p * q.d[qclass(i)];
    }
    static __device__ __forceinline__ int16_t round_nearest(float v, const Q& q, int i) {
        unsigned short r;
        asm("cvt.rni.sat.s16.f32 %0, %1;" : "=h"(r) : "f"(v * q.inv[qclass(i)]));
        return (int16_t)r;
    }
    // floor(v / d + u) with u uniform in [0, 1): the 16 random bits form 1 + u in FP32
    static __device__ __forceinline__ int16_t round_stochastic(float v, uint32_t r, const Q& q, int i) {
        const float u = __uint_as_float(0x3F800000u | ((r & 0xFFFFu) << 7)) - 1.0f;
        unsigned short o;
        asm("cvt.rmi.sat.s16.f32 %0, %1;" : "=h"(o) : "f"(fmaf(v, q.inv[qclass(i)], u)));
        return (int16_t)o;
    }
    static __device__ __forceinline__ void store(int16_t* p, float v, const Q& q, int i) { *p = round_nearest(v, q, i); }
    static __device__ __forceinline__ void store_sr(int16_t* p, float v, uint32_t r, const Q& q, int i) {
        *p = round_stochastic(v, r, q, i);
    }
    static __device__ __forceinline__ bool at_limit(const int16_t* p) {
        const int16_t v = *p;
        return v == (int16_t)-32768 || v == (int16_t)32767;
    }
};

// Counter-based 32-bit mixer for the stochastic-rounding bits of one population store: a function
// of (sample, in-sample offset, step) only, so runs reproduce.  It is the xor-shift-multiply
// integer hash "lowbias32" (shift 16, multiply, shift 15, multiply, shift 16) with the constants
// published by C. Wellons's hash-prospector search.
__device__ __forceinline__ uint32_t mix32(uint32_t x) {
    x ^= x >> 16;
    x *= 0x7feb352dU;
    x ^= x >> 15;
    x *= 0x846ca68bU;
    x ^= x >> 16;
    return x;
}

// Division in the FP32 moments: 1 = the fast reciprocal-and-multiply form (within 2 ulp of the small
// correction 1/rho - 1), 0 = IEEE division.  Measured on the cluster scheme (FP32 cylinder, 9 x 440 x
// 82; BF16 channel samples of the uneven batch): 57.9 / 53.7 against 53.5 / 50.0 GLUPS.
#ifndef UQLB_FAST_DIV_F32
#define UQLB_FAST_DIV_F32 1
#endif
// Moments of shifted populations: drho, j = sum c_i g_i and u = j / rho = j + j (1/rho - 1).
template <typename C>
__device__ __forceinline__ void moments(const C g[9], C& drho, C& jx, C& jy, C& ux, C& uy) {
    drho = ((g[0] + g[1]) + (g[2] + g[3])) + ((g[4] + g[5]) + (g[6] + g[7])) + g[8];
    jx = (g[1] - g[3]) + (g[5] - g[6]) + (g[8] - g[7]);
    jy = (g[2] - g[4]) + (g[5] - g[7]) + (g[6] - g[8]);
#if UQLB_FAST_DIV_F32
    C d;  // 1/rho - 1
    if constexpr (sizeof(C) == 4)
        d = __fdividef(-drho, C(1) + drho);
    else
        d = -drho / (C(1) + drho);
#else
    const C d = -drho / (C(1) + drho);  // 1/rho - 1
#endif
    ux = fma(jx, d, jx);
    uy = fma(jy, d, jy);
}

// Coefficient of the linear equilibrium term, L_i = 3 w_i, written on the momentum:
// rho w_i 3 c_i.u = L_i c_i.j.  The diagonal value is one unit in the last place below 1/12 so
// that 2 L_1 + 4 L_5 = 1 holds exactly in the arithmetic type; the equilibrium then carries
// exactly the momentum j.  With the rounded 3 w_i the sum is 1 + 3e-8 in FP32, and the BGK
// update would add omega * 3e-8 of relative momentum at every step of every node.
template <typename C>
__device__ __forceinline__ C lin(int i);
template <>
__device__ __forceinline__ float lin<float>(int i) {
    return i == 0 ? 0.0f : (i <= 4 ? 0x1.555556p-2f : 0x1.555554p-4f);
}
template <>
__device__ __forceinline__ double lin<double>(int i) {
    return i == 0 ? 0.0 : (i <= 4 ? 0x1.5555555555555p-2 : 0x1.5555555555556p-4);
}

// BGK relaxation of shifted populations towards the shifted equilibrium, in place:
//   g_i^eq = w_i (drho + 4.5 (c_i.j)(c_i.u) - 1.5 j.u) + L_i c_i.j
// (Eq. equilibrium times rho, with rho u = j), g_i* = g_i + omega (g_i^eq - g_i).
// Opposite directions share the even part A = w_i (drho + 4.5 (c_i.j)(c_i.u) - 1.5 j.u) and
// differ in the sign of the odd part, so each pair (i, opp(i)) is evaluated once:
// g_i^eq = fma(L_i, c_i.j, A), g_opp^eq = fma(-L_i, c_i.j, A) (the same roundings as
// evaluating every direction on its own).
template <typename C>
__device__ __forceinline__ void bgk(C g[9], C omega, C drho, C jx, C jy, C ux, C uy) {
    const C ju15 = C(1.5) * (jx * ux + jy * uy);
    g[0] = fma(omega, wgt<C>(0) * (drho - ju15) - g[0], g[0]);
#pragma unroll
    for (int i : {1, 2, 5, 6}) {
        const int o = opp(i);
        const C cj = C(cx(i)) * jx + C(cy(i)) * jy;
        const C cu = C(cx(i)) * ux + C(cy(i)) * uy;
        const C A = wgt<C>(i) * (drho + C(4.5) * cj * cu - ju15);
        const C gi = fma(lin<C>(i), cj, A);
        const C go = fma(-lin<C>(i), cj, A);
        g[i] = fma(omega, gi - g[i], g[i]);
        g[o] = fma(omega, go - g[o], g[o]);
    }
}

// ---- Two nodes at once in packed FP32 (sm_100+ f32x2 arithmetic) ---------------------------
// A 64-bit register holds one value of node a (low half) and of node b (high half); each packed
// add / sub / mul / fma rounds both halves as the scalar instruction does.
using f2 = unsigned long long;
__device__ __forceinline__ f2 pk(float lo, float hi) {
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void upk(f2 v, float& lo, float& hi) { asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v)); }
__device__ __forceinline__ f2 add2(f2 a, f2 b) {
    f2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 sub2(f2 a, f2 b) {
    f2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 mul2(f2 a, f2 b) {
    f2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) {
    f2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ f2 splat(float c) { return pk(c, c); }

// Relaxation constants of the packed collision for one relaxation rate omega.  The BGK update is
// written as g_i* = (1 - omega) g_i + omega g_i^eq, with omega folded into the equilibrium's
// coefficients: omega w_i for the even part and omega L_i for the odd part.  The odd coefficients
// keep 2 omega L_1 + 4 omega L_5 = omega exactly (ol5 = (omega - 2 ol1) / 4, an exact difference and an
// exact quarter), so the relaxation carries exactly the momentum omega j, as the unfolded form does
// with 2 L_1 + 4 L_5 = 1; 1 - omega is exact for omega in [0.5, 2] (tau <= 2).
struct PackedBGK {
    f2 omc, ow0, ow1, ow5, ol1, ol5, nl1, nl5;  // nl = -ol
};
__device__ __forceinline__ PackedBGK packed_bgk(float omega) {
    PackedBGK k;
    k.omc = splat(1.0f - omega);
    k.ow0 = splat(omega * wgt<float>(0));
    k.ow1 = splat(omega * wgt<float>(1));
    k.ow5 = splat(omega * wgt<float>(5));
    const float ol1 = omega * lin<float>(1);
    k.ol1 = splat(ol1);
    const float ol5 = (omega - 2.0f * ol1) * 0.25f;
    k.ol5 = splat(ol5);
    k.nl1 = splat(-ol1);
    k.nl5 = splat(-ol5);
    return k;
}

// The BGK collision of two nodes a and b in packed arithmetic (the formulas of moments() and bgk(),
// with omega folded into the equilibrium as PackedBGK describes; the operation order is fixed here, so
// results agree with the scalar path to round-off).  g[i] holds population i of node a (low half) and
// of node b (high half); usq (when non-null) receives u.u of both nodes.
//   drho = sum g_i, j = sum c_i g_i (with a = g5 - g7, b = g6 - g8 shared by jx and jy), u = j + j d,
//   X = drho - 1.5 j.u, and per pair of opposite directions (i, opp i):
//   omega A = omega w_i (X + 4.5 (c_i.j)(c_i.u)),  g_i* = (1 - omega) g_i + (omega A + omega L_i c_i.j),
//   g_opp* = (1 - omega) g_opp + (omega A - omega L_i c_i.j);  rest: g_0* = (1 - omega) g_0 + omega w_0 X.
__device__ __forceinline__ void collide_packed(f2 (&g)[9], const PackedBGK& k, f2* usq) {
    const f2 drho =
        add2(add2(add2(add2(g[0], g[1]), add2(g[2], g[3])), add2(add2(g[4], g[5]), add2(g[6], g[7]))), g[8]);
    const f2 a = sub2(g[5], g[7]), b = sub2(g[6], g[8]);
    const f2 jx = add2(sub2(g[1], g[3]), sub2(a, b));
    const f2 jy = add2(sub2(g[2], g[4]), add2(a, b));
    float da, db;
    upk(drho, da, db);
    // 1/rho - 1 per node; the fast division (reciprocal and multiply, within 2 ulp) is exact enough
    // for this small correction (|drho| << 1: its error is ~1e-7 of ~1e-4 of u) and saves the
    // IEEE division's refinement steps
    const f2 d = pk(__fdividef(-da, 1.0f + da), __fdividef(-db, 1.0f + db));
    const f2 ux = fma2(jx, d, jx), uy = fma2(jy, d, jy);
    if (usq != nullptr) *usq = fma2(uy, uy, mul2(ux, ux));
    const f2 X = fma2(splat(-1.5f), fma2(jy, uy, mul2(jx, ux)), drho);
    const f2 ux45 = mul2(splat(4.5f), ux), uy45 = mul2(splat(4.5f), uy);
    g[0] = fma2(g[0], k.omc, mul2(k.ow0, X));
#pragma unroll
    for (int i : {1, 2, 5, 6}) {
        const int o = opp(i);
        f2 cj, cu, ow, ol, nl;
        if (i == 1) {
            cj = jx;
            cu = ux45;
        } else if (i == 2) {
            cj = jy;
            cu = uy45;
        } else if (i == 5) {
            cj = add2(jx, jy);
            cu = add2(ux45, uy45);
        } else {
            cj = sub2(jy, jx);
            cu = sub2(uy45, ux45);
        }
        ow = i <= 4 ? k.ow1 : k.ow5;
        ol = i <= 4 ? k.ol1 : k.ol5;
        nl = i <= 4 ? k.nl1 : k.nl5;
        const f2 oA = mul2(ow, fma2(cj, cu, X));
        g[i] = fma2(g[i], k.omc, fma2(ol, cj, oA));
        g[o] = fma2(g[o], k.omc, fma2(nl, cj, oA));
    }
}

// collide_packed() on two nodes held as separate arrays.
__device__ __forceinline__ void collide_pair(float (&ga)[9], float (&gb)[9], const PackedBGK& omega, float* usq_a,
                                             float* usq_b) {
    f2 g[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) g[i] = pk(ga[i], gb[i]);
    f2 q;
    collide_packed(g, omega, usq_a != nullptr ? &q : nullptr);
    if (usq_a != nullptr) upk(q, *usq_a, *usq_b);
#pragma unroll
    for (int i = 0; i < 9; ++i) upk(g[i], ga[i], gb[i]);
}

// Two nodes collided one after the other in scalar FP32 (moments() and bgk() of each), the same
// formulas as collide_packed() issued on the scalar FP32 pipe; usq_a/usq_b (when non-null) receive u.u.
__device__ __forceinline__ void collide_pair_scalar(float (&ga)[9], float (&gb)[9], float omega, float* usq_a,
                                                    float* usq_b) {
    float drho, jx, jy, ux, uy;
    moments(ga, drho, jx, jy, ux, uy);
    if (usq_a != nullptr) *usq_a = fmaf(uy, uy, ux * ux);
    bgk(ga, omega, drho, jx, jy, ux, uy);
    moments(gb, drho, jx, jy, ux, uy);
    if (usq_b != nullptr) *usq_b = fmaf(uy, uy, ux * ux);
    bgk(gb, omega, drho, jx, jy, ux, uy);
}

// Obstacle bitmask lookup: bit (x & 31) of word y * words + (x >> 5).
__device__ __forceinline__ bool mask_solid(const uint32_t* m, int words, int x, int y) {
    return (__ldg(m + (int64_t)y * words + (x >> 5)) >> (x & 31)) & 1u;
}

}  // namespace uqlb
