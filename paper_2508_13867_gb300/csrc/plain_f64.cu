// Plain per-sample FP64 path: the unbatched, unfused comparator of the batched ensemble.
//
// One sample at a time, one launch per time step on two full lattices f[9][ny][nx] (FP64,
// unshifted populations), collide-then-push streaming exactly as written in Sec. 3
// (f*(x) = f - (f - f^eq)/tau; f(x + c_i, t + 1) = f*_i(x, t)), boundary rules applied where a
// population leaves through a boundary link (same rules as the batched kernels), and every
// quantity of interest computed by its own kernels after the step that produced the state.
#include <cmath>

#include "d2q9.cuh"
#include "uqlb_internal.h"

namespace uqlb {

namespace {

constexpr int kBlock = 256;

__device__ __forceinline__ double feq_d(int i, double rho, double ux, double uy) {
    const double cu = cx(i) * ux + cy(i) * uy;
    return wgt<double>(i) * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * (ux * ux + uy * uy));
}

__global__ void plain_init(PlainSample p, double* f, const uint8_t* solid) {
    const int64_t n = (int64_t)p.nx * p.ny;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(k % p.nx), y = (int)(k / p.nx);
        double rho = 1.0, ux = 0.0, uy = 0.0;
        if (p.kind == UQLB_CASE_TGV) {
            const double kx = 2.0 * M_PI / p.nx, ky = 2.0 * M_PI / p.ny;
            ux = p.u0 * sin(kx * x) * cos(ky * y) + p.amp2 * sin(2 * kx * x) * cos(2 * ky * y) +
                 p.amp3 * sin(3 * kx * x) * cos(3 * ky * y);
            uy = -p.u0 * cos(kx * x) * sin(ky * y) - p.amp2 * cos(2 * kx * x) * sin(2 * ky * y) -
                 p.amp3 * cos(3 * kx * x) * sin(3 * ky * y);
            rho = 1.0 + 3.0 * 0.25 * p.u0 * p.u0 * (cos(2 * kx * x) + cos(2 * ky * y));
        }
        if (solid[k]) ux = uy = 0.0;
        for (int i = 0; i < 9; ++i) f[i * n + k] = feq_d(i, rho, ux, uy);
    }
}

__device__ __forceinline__ double inflow_d(const PlainSample& p, double yy, int t) {
    double ramp = 1.0;
    if (p.ramp_steps > 0.0 && (double)t < p.ramp_steps) ramp = 0.5 * (1.0 - cos(M_PI * t / p.ramp_steps));
    const double H = p.ny;
    return 4.0 * p.uin_max * ramp * yy * (H - yy) / (H * H);
}

// One time step: collide at x, push f*_i to x + c_i (or apply the boundary rule of that link).
__global__ void plain_step(PlainSample p, const double* __restrict__ fin, double* __restrict__ fout,
                           const uint8_t* __restrict__ solid, int t) {
    const int64_t n = (int64_t)p.nx * p.ny;
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= n || solid[k]) return;
    const int x = (int)(k % p.nx), y = (int)(k / p.nx);
    double f[9], rho = 0.0, jx = 0.0, jy = 0.0;
    for (int i = 0; i < 9; ++i) {
        f[i] = fin[i * n + k];
        rho += f[i];
        jx += cx(i) * f[i];
        jy += cy(i) * f[i];
    }
    const double ux = jx / rho, uy = jy / rho;
    for (int i = 0; i < 9; ++i) f[i] = f[i] - p.omega * (f[i] - feq_d(i, rho, ux, uy));
    for (int i = 0; i < 9; ++i) {
        int dx = x + cx(i), dy = y + cy(i);
        const int o = opp(i);
        if (p.kind == UQLB_CASE_TGV) {
            dx = (dx + p.nx) % p.nx;
            dy = (dy + p.ny) % p.ny;
            fout[i * n + (int64_t)dy * p.nx + dx] = f[i];
        } else if (dy < 0 || dy >= p.ny) {
            fout[o * n + k] = f[i];
        } else if (dx < 0) {
            const double yy = y + 0.5 - 0.5 * cy(o);
            fout[o * n + k] = f[i] + 6.0 * wgt<double>(o) * cx(o) * inflow_d(p, yy, t);
        } else if (dx >= p.nx) {
            const double cu = cx(o) * ux + cy(o) * uy;
            fout[o * n + k] = -f[i] + 2.0 * wgt<double>(o) * (1.0 + 4.5 * cu * cu - 1.5 * (ux * ux + uy * uy));
        } else if (solid[(int64_t)dy * p.nx + dx]) {
            fout[o * n + k] = f[i];
        } else {
            fout[i * n + (int64_t)dy * p.nx + dx] = f[i];
        }
    }
}

// Per-block partial sums of (K, mass, mx, my, Fx, Fy, bad) of the state f at time t; the
// forces use the bounce-back populations, which are the post-collision values of step t - 1.
__global__ void plain_qoi(PlainSample p, const double* __restrict__ f, const uint8_t* __restrict__ solid,
                          double* partials, double* fields, int want_force) {
    __shared__ double sm[kBlock / 32][7];
    const int64_t n = (int64_t)p.nx * p.ny;
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    double v[7] = {0, 0, 0, 0, 0, 0, 0};
    if (k < n) {
        double ux = 0.0, uy = 0.0;
        if (!solid[k]) {
            const int x = (int)(k % p.nx), y = (int)(k / p.nx);
            double rho = 0.0, jx = 0.0, jy = 0.0;
            for (int i = 0; i < 9; ++i) {
                const double fi = f[i * n + k];
                rho += fi;
                jx += cx(i) * fi;
                jy += cy(i) * fi;
            }
            ux = jx / rho;
            uy = jy / rho;
            v[0] = ux * ux + uy * uy;
            v[1] = rho;
            v[2] = rho * ux;
            v[3] = rho * uy;
            v[6] = (!(rho > 0.0) || !isfinite(ux) || !isfinite(uy)) ? 1.0 : 0.0;
            if (want_force) {
                for (int i = 1; i < 9; ++i) {
                    const int xn = x + cx(i), yn = y + cy(i);
                    if (xn >= 0 && xn < p.nx && yn >= 0 && yn < p.ny && solid[(int64_t)yn * p.nx + xn]) {
                        const double fs = f[opp(i) * n + k];
                        v[4] += 2.0 * cx(i) * fs;
                        v[5] += 2.0 * cy(i) * fs;
                    }
                }
            }
        }
        if (fields != nullptr) {
            fields[k] = ux;
            fields[n + k] = uy;
        }
    }
    for (int q = 0; q < 7; ++q)
        for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
    if ((threadIdx.x & 31) == 0)
        for (int q = 0; q < 7; ++q) sm[threadIdx.x >> 5][q] = v[q];
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int q = 0; q < 7; ++q) {
            double s = 0.0;
            for (int w = 0; w < kBlock / 32; ++w) s += sm[w][q];
            partials[(int64_t)blockIdx.x * 7 + q] = s;
        }
    }
}

// Second pass: sum the block partials in order and write the sample's scalars.
__global__ void plain_qoi_total(PlainSample p, const double* partials, int nblocks, int t,
                                double* qoi_row, double* series_slot, double* fields_k, double* cd_out) {
    if (threadIdx.x != 0) return;
    double s[7] = {0, 0, 0, 0, 0, 0, 0};
    for (int b = 0; b < nblocks; ++b)
        for (int q = 0; q < 7; ++q) s[q] += partials[(int64_t)b * 7 + q];
    const double K = s[0] * p.u_ref_inv2;
    if (series_slot != nullptr) *series_slot = (p.kind == UQLB_CASE_TGV) ? K : s[4] * p.force_norm;
    if (cd_out != nullptr) *cd_out = s[4] * p.force_norm;
    if (fields_k != nullptr) *fields_k = K;
    if (qoi_row != nullptr) {
        qoi_row[UQLB_QOI_K] = K;
        qoi_row[UQLB_QOI_MASS] = s[1];
        qoi_row[UQLB_QOI_MOMX] = s[2];
        qoi_row[UQLB_QOI_MOMY] = s[3];
        qoi_row[UQLB_QOI_CD] = s[4] * p.force_norm;
        qoi_row[UQLB_QOI_CL] = s[5] * p.force_norm;
        qoi_row[UQLB_QOI_STEPS] = (double)t;
        qoi_row[UQLB_QOI_STATUS] = s[6] > 0.0 ? (double)UQLB_ERR_UNSTABLE : 0.0;
    }
}

}  // namespace

cudaError_t plain_run_sample(const PlainSample& p, double* f_a, double* f_b, uint8_t* solid,
                             double* partials, int64_t qoi_every, double* fields, double* qoi_row,
                             double* series_row, cudaStream_t s) {
    const int64_t n = (int64_t)p.nx * p.ny;
    const int blocks = (int)((n + kBlock - 1) / kBlock);
    plain_init<<<blocks, kBlock, 0, s>>>(p, f_a, solid);
    const bool channel = p.kind == UQLB_CASE_CHANNEL;
    const int want_force = channel && p.cyl_r > 0.0;
    if (!channel && qoi_every > 0 && series_row != nullptr) {
        plain_qoi<<<blocks, kBlock, 0, s>>>(p, f_a, solid, partials, nullptr, 0);
        plain_qoi_total<<<1, 32, 0, s>>>(p, partials, blocks, 0, nullptr, series_row, nullptr, nullptr);
    }
    double* cur = f_a;
    double* nxt = f_b;
    int t = 0;
    for (; t < p.steps; ++t) {
        plain_step<<<blocks, kBlock, 0, s>>>(p, cur, nxt, solid, t);
        double* tmp = cur;
        cur = nxt;
        nxt = tmp;
        const int tn = t + 1;
        if (qoi_every > 0 && tn % qoi_every == 0 && series_row != nullptr) {
            plain_qoi<<<blocks, kBlock, 0, s>>>(p, cur, solid, partials, nullptr, want_force);
            const int64_t col = channel ? tn / qoi_every - 1 : tn / qoi_every;
            plain_qoi_total<<<1, 32, 0, s>>>(p, partials, blocks, tn, nullptr, series_row + col, nullptr, nullptr);
        }
    }
    plain_qoi<<<blocks, kBlock, 0, s>>>(p, cur, solid, partials, fields, want_force);
    plain_qoi_total<<<1, 32, 0, s>>>(p, partials, blocks, t, qoi_row, nullptr,
                                     fields != nullptr ? fields + 2 * n : nullptr, nullptr);
    return cudaGetLastError();
}

}  // namespace uqlb
