// Batched D2Q9 BGK ensemble kernels for sm_103a (arXiv 2508.13867, Sec. 3 and Sec. 7).
//
// Included by one translation unit per population storage type (lbm_<type>.cu), which
// instantiates every kernel for its type and exports the launchers as a StorageOps table.
//
// All samples of an ensemble live in one arena, sample-major, and every kernel addresses a
// population as arena[f_off(s) + i * plane(s) + y * pitch(s) + x], g_i = f_i - w_i.  One-step runs
// keep population planes (plane = cols * ny, pitch = cols); multi-step runs keep each row's nine
// populations together (plane = cols, pitch = 9 cols), so a row is one contiguous block.
// One-step scheme (step_kernel, persistent_kernel): the lattice is updated in place in AA order:
// an even step reads and writes the nine populations of its own node (writing post-collision g_i
// to slot opp(i)); an odd step reads the incoming populations from the neighbours' slots and
// writes its outgoing populations into the neighbours' slots.  Every memory location is read and
// then written by exactly one thread per step, so no second lattice and no intra-step
// synchronisation are needed.  Multi-step schemes (periodic batches; strip2_kernel and strip3_kernel
// on row strips, step2_kernel on tiles): two lattices in natural order, each launch collides,
// streams through shared memory, collides again (once or twice) and pushes into the other lattice.
// Boundary rules are applied where a population crosses a boundary link:
//   periodic (TGV, Sec. 8.2): wrap-around neighbours;
//   wall / obstacle (Sec. 8.1 no-slip): halfway bounce-back;
//   inlet (x = 0 face): moving-wall bounce-back with the parabolic profile at the link midpoint;
//   outlet (x = nx face): anti-bounce-back at rho = 1 with the outlet node's velocity.
// Quantities of interest are reduced in the same kernel: K(t) from the pre-collision moments
// and drag/lift by momentum exchange from the post-collision populations; per-tile partial
// sums (FP64) are combined in a fixed order by the last tile of each sample to finish.
#include <algorithm>
#include <cmath>
#include <type_traits>

#include "d2q9.cuh"
#include "lbm_common.cuh"

#pragma once

namespace uqlb {

namespace {

// Sample index j (in table order) of a global tile index.
__device__ __forceinline__ int tile_sample(const KParams& p, int tile, int nact) {
    if (p.uniform_tiles > 0) return tile / p.uniform_tiles;
    int lo = 0, hi = nact - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (p.samples[mid].tile_base <= tile)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// Quanta of sample j (table order) for the fixed-point storage; an empty value for other formats.
template <typename S>
__device__ __forceinline__ typename Storage<S>::Q quanta_of(const KParams& p, int j) {
    typename Storage<S>::Q q{};
    if constexpr (std::is_same<typename Storage<S>::Q, Quanta>::value) {
        const InitDev& in = p.init[j];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            q.d[c] = __ldg(&in.quanta[c]);
            q.inv[c] = __ldg(&in.inv_quanta[c]);
        }
    }
    return q;
}

// Number of samples with steps > t (the table is ordered by descending steps).
__device__ __forceinline__ int active_samples(const KParams& p, int t) {
    int lo = 0, hi = p.nsamples;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (p.steps_sorted[mid] > t)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

// Link classes of the channel case, checked in this order.
enum LinkClass { kInterior = 0, kWall = 1, kInlet = 2, kOutlet = 3, kSolid = 4 };

__device__ __forceinline__ int classify(const SampleDev& sp, const uint32_t* mask, int xn, int yn) {
    if (yn < 0 || yn >= sp.ny) return kWall;
    if (xn < 0) return kInlet;
    if (xn >= sp.nx) return kOutlet;
    if (mask != nullptr && mask_solid(mask, mask_words(sp), xn, yn)) return kSolid;
    return kInterior;
}

__device__ __forceinline__ float cospi_c(float a) { return cospif(a); }
__device__ __forceinline__ double cospi_c(double a) { return cospi(a); }

// Inflow velocity at height yy (walls at 0 and ny) at step t, Sec. 8.1 profile and ramp.  The
// ramp is evaluated in the compute type: FP64 runs at a small fraction of the FP32 rate on this
// part, and a warp holding an inlet node would otherwise wait on six FP64 cosines per step.
template <typename C>
__device__ __forceinline__ C inflow(const SampleDev& sp, C yy, int t) {
    C ramp = C(1);
    if (sp.ramp_steps > 0.0 && (double)t < sp.ramp_steps)
        ramp = C(0.5) * (C(1) - cospi_c(C(t) / C(sp.ramp_steps)));
    const C H = C(sp.ny);
    return C(4) * C(sp.uin_max) * ramp * yy * (H - yy) / (H * H);
}

// ---- Bouzidi linear interpolated bounce-back on the obstacle (Sec. 8.1 cylinder surface) ----
// A link from fluid node x along c_i into the obstacle meets the circle at the fraction q of its
// length; the population returning to x is 2q g*_i(x) + (1 - 2q) g_i(x, t+1) for q < 1/2 and
// g*_i(x) / (2q) + (1 - 1/(2q)) g*_ibar(x) for q >= 1/2 (weights sum to 1, so the shifted
// g = f - w obey the same rule).  In the in-place AA layout the collision writes the part it can
// form locally into the node's own bounce-back slot opp(i) (the whole value for q >= 1/2, 2q g*_i
// below), the gather of the next step adds (1 - 2q) times the streamed g_i, and the raw g*_i is
// parked in slot i of the obstacle node x + c_i, which no thread reads or writes otherwise (it
// serves the force).

// q of the link from (x, y) along c_i: the entry root of |P + s c_i - C|^2 = r^2 (P the node
// centre), as s = 2 cc / (sqrt(b^2 - 4 a cc) - b), free of cancellation since b < 0 on a link
// that enters the circle.
template <typename C>
__device__ __forceinline__ C link_q(const InitDev& in, int x, int y, int i) {
    const double px = (double)x + 0.5 - in.cyl_cx, py = (double)y + 0.5 - in.cyl_cy;
    const C cc = (C)(px * px + py * py - in.cyl_r * in.cyl_r);
    const C b = C(2) * (C(cx(i)) * (C)px + C(cy(i)) * (C)py);
    const C a = C(cx(i) * cx(i) + cy(i) * cy(i));
    return C(2) * cc / (sqrt(b * b - C(4) * a * cc) - b);
}

// Directions i (bit i) of node (x, y) whose neighbour x + c_i is an obstacle node.
__device__ __forceinline__ uint32_t obstacle_links(const SampleDev& sp, const InitDev& in, const uint32_t* mask,
                                                   int x, int y) {
    if (x < in.bbox[0] || x > in.bbox[1] || y < in.bbox[2] || y > in.bbox[3]) return 0u;
    uint32_t m = 0u;
#pragma unroll
    for (int i = 1; i < 9; ++i) {
        const int xn = x + cx(i), yn = y + cy(i);
        if (xn >= 0 && xn < sp.nx && yn >= 0 && yn < sp.ny && mask_solid(mask, mask_words(sp), xn, yn))
            m |= 1u << i;
    }
    return m;
}

// Gather side: g[opp(i)] holds what the collision left in the bounce-back slot.
template <typename C>
__device__ __forceinline__ void bouzidi_complete(const InitDev& in, int x, int y, uint32_t links, C (&g)[9]) {
#pragma unroll
    for (int i = 1; i < 9; ++i) {
        if (links >> i & 1u) {
            const C q = link_q<C>(in, x, y, i);
            if (q < C(0.5)) g[opp(i)] += (C(1) - C(2) * q) * g[i];
        }
    }
}

// Collision side: the value written to the bounce-back slot opp(i) from the post-collision g*.
template <typename C>
__device__ __forceinline__ C bouzidi_local(const InitDev& in, int x, int y, int i, const C (&g)[9]) {
    const C q = link_q<C>(in, x, y, i);
    return q < C(0.5) ? C(2) * q * g[i] : (g[i] + (C(2) * q - C(1)) * g[opp(i)]) / (C(2) * q);
}

// Shifted incoming population of direction i at node (x, y) for the stream (tp -> tp + 1),
// given the slot layout left by an even step at time tp: g_i*(z) sits at (z, slot opp(i)).
// ub: velocity of the outlet node at time tp.
template <typename S>
__device__ __forceinline__ typename Storage<S>::C read_incoming(
    const S* base, const SampleDev& sp, const uint32_t* mask, int x, int y, int i, int tp,
    typename Storage<S>::C ubx, typename Storage<S>::C uby, bool chan, const typename Storage<S>::Q& qz) {
    using C = typename Storage<S>::C;
    const int64_t plane = sp.plane;
    const int pitch = sp.pitch;
    int sx = x - cx(i), sy = y - cy(i);
    if (!chan) {
        sx = sx < 0 ? sx + sp.nx : (sx >= sp.nx ? sx - sp.nx : sx);
        sy = sy < 0 ? sy + sp.ny : (sy >= sp.ny ? sy - sp.ny : sy);
        return Storage<S>::load(base + opp(i) * plane + (int64_t)sy * pitch + sx, qz, i);
    } else {
        const int cls = classify(sp, mask, sx, sy);
        const int64_t own = (int64_t)y * pitch + x;
        if (cls == kInterior) return Storage<S>::load(base + opp(i) * plane + (int64_t)sy * pitch + sx, qz, i);
        const C mine = Storage<S>::load(base + i * plane + own, qz, i);  // g_opp(i)*(x, tp)
        if (cls == kWall || cls == kSolid) return mine;
        if (cls == kInlet) {
            const C yy = C(y) + C(0.5) - C(0.5) * C(cy(i));
            return mine + C(6) * wgt<C>(i) * C(cx(i)) * inflow<C>(sp, yy, tp);
        }
        // outlet: g_i = -g_opp(i)* + w_i (9 (c_i.u)^2 - 3 u.u)
        const C cu = C(cx(i)) * ubx + C(cy(i)) * uby;
        return -mine + wgt<C>(i) * (C(9) * cu * cu - C(3) * (ubx * ubx + uby * uby));
    }
}

// Block-wide deterministic sum of NV doubles; result valid in thread 0.
template <int NV, int NT>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* smem) {
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
    }
    const int warp = tid >> 5, lane = tid & 31;
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) smem[warp * NV + k] = v[k];
    }
    __syncthreads();
    if (tid == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double s = 0.0;
            for (int w = 0; w < NT / 32; ++w) s += smem[w * NV + k];
            v[k] = s;
        }
    }
    __syncthreads();
}

// Publish this tile's partial sums; returns true in every thread of the block that finished
// the sample's last tile, after which `tot` holds the fixed-order total in thread 0.
template <int NV, int NT>
__device__ __forceinline__ bool tile_reduce_last(const KParams& p, const SampleDev& sp, int j,
                                                 int tile, double (&v)[NV], double (&tot)[NV],
                                                 double* smem, int* sflag) {
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    block_sum<NV, NT>(v, smem);
    if (tid == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) p.partials[(int64_t)tile * NV + k] = v[k];
        __threadfence();
        const int prev = atomicAdd(p.counters + j, 1);
        *sflag = (prev == sp.tiles - 1);
    }
    __syncthreads();
    const bool last = *sflag != 0;
    if (last) {
        __threadfence();
        double acc[NV];
#pragma unroll
        for (int k = 0; k < NV; ++k) acc[k] = 0.0;
        for (int q = tid; q < sp.tiles; q += NT) {
#pragma unroll
            for (int k = 0; k < NV; ++k) acc[k] += __ldcg(p.partials + (int64_t)(sp.tile_base + q) * NV + k);
        }
        block_sum<NV, NT>(acc, smem);
        if (tid == 0) {
#pragma unroll
            for (int k = 0; k < NV; ++k) tot[k] = acc[k];
            p.counters[j] = 0;
        }
    }
    __syncthreads();
    return last;
}

// ------------------------------------------------------------------------------------------
// Initial state: equilibrium of the initial macroscopic field (Sec. 8.2 TGV, Sec. 8.1 rest).
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ void sincospi_c(float a, float* s, float* c) { sincospif(a, s, c); }
__device__ __forceinline__ void sincospi_c(double a, double* s, double* c) { sincospi(a, s, c); }

template <typename S>
__global__ void __launch_bounds__(256) init_kernel(KParams p, int64_t total_tiles, int tile_rows, int tile_cols) {
    using C = typename Storage<S>::C;
    S* arena = static_cast<S*>(p.arena);
    for (int64_t tile = blockIdx.x; tile < total_tiles; tile += gridDim.x) {
        const int j = tile_sample(p, (int)tile, p.nsamples);
        const SampleDev& sp = p.samples[j];
        const typename Storage<S>::Q qz = quanta_of<S>(p, j);
        const int lt = (int)tile - sp.tile_base;
        const int y0 = (lt / sp.tiles_x) * tile_rows;
        if (tile == sp.tile_base && threadIdx.x == 0) {
            p.counters[j] = 0;
            p.done[sp.slot] = 0;
            p.steps_run[sp.slot] = sp.steps;
            p.cd_prev[sp.slot] = NAN;
            p.streak[sp.slot] = 0;
            if (p.sel != nullptr) p.sel[sp.slot] = 0;  // the initial state is in the first lattice
        }
        for (int q = threadIdx.x; q < tile_rows * tile_cols; q += blockDim.x) {
            const int x = (lt % sp.tiles_x) * tile_cols + (q % tile_cols);
            const int y = y0 + q / tile_cols;
            if (x >= sp.nx || y >= sp.ny) continue;
            // The analytic field and its equilibrium in the storage's compute type (FP64 for FP64
            // storage, FP32 otherwise); the density enters as drho = rho - 1, so no 1 + small
            // cancellation occurs in FP32.
            C drho = C(0), ux = C(0), uy = C(0);
            if (sp.kind == UQLB_CASE_TGV) {
                const InitDev& in = p.init[j];
                const C u0 = (C)in.u0, a2 = (C)in.amp2, a3 = (C)in.amp3;
                C s1x, c1x, s1y, c1y;
                sincospi_c(C(2 * x) / C(sp.nx), &s1x, &c1x);
                sincospi_c(C(2 * y) / C(sp.ny), &s1y, &c1y);
                const C s2x = C(2) * s1x * c1x, c2x = C(2) * c1x * c1x - C(1);
                const C s2y = C(2) * s1y * c1y, c2y = C(2) * c1y * c1y - C(1);
                const C s3x = s1x * (C(3) - C(4) * s1x * s1x), c3x = c1x * (C(4) * c1x * c1x - C(3));
                const C s3y = s1y * (C(3) - C(4) * s1y * s1y), c3y = c1y * (C(4) * c1y * c1y - C(3));
                ux = u0 * s1x * c1y + a2 * s2x * c2y + a3 * s3x * c3y;
                uy = -u0 * c1x * s1y - a2 * c2x * s2y - a3 * c3x * s3y;
                drho = C(0.75) * u0 * u0 * (c2x + c2y);  // 3 p, p = u0^2 / 4 (cos 2kx + cos 2ky)
            } else if (sp.kind == UQLB_CASE_TGV_PERTURBED) {
                // Sec. 8.3: base mode 2 with amplitude U = u0 + eps(x, y), perturbation modes 4
                const InitDev& in = p.init[j];
                C s2x, c2x, s2y, c2y;
                sincospi_c(C(4 * x) / C(sp.nx), &s2x, &c2x);
                sincospi_c(C(4 * y) / C(sp.ny), &s2y, &c2y);
                const C s4x = C(2) * s2x * c2x, c4x = C(2) * c2x * c2x - C(1);
                const C s4y = C(2) * s2y * c2y, c4y = C(2) * c2y * c2y - C(1);
                const C eps = (C)in.pert[0] * s4x * s4y + (C)in.pert[1] * s4x * c4y + (C)in.pert[2] * c4x * s4y +
                              (C)in.pert[3] * c4x * c4y;
                const C U = (C)in.u0 + C(0.25) * eps;
                ux = -U * c2x * s2y;
                uy = U * s2x * c2y;
                drho = -C(0.75) * U * U * (c4x + c4y);
            }
            const C usq = ux * ux + uy * uy, rho = C(1) + drho;
            S* base = arena + sp.f_off + (int64_t)y * sp.pitch + x;
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                const C cu = C(cx(i)) * ux + C(cy(i)) * uy;
                const C w = wgt<C>(i);
                const C g = w * drho + w * rho * (C(3) * cu + C(4.5) * cu * cu - C(1.5) * usq);
                Storage<S>::store(base + i * sp.plane, g, qz, i);
            }
        }
    }
}

// ------------------------------------------------------------------------------------------
// Fused collide-stream-boundary-QoI step (one launch per time step).
// ------------------------------------------------------------------------------------------

// Periodic neighbourhood of a node: wrapped columns x-1, x, x+1 and row offsets of y-1, y, y+1,
// indexed by c + 1.  In-sample offsets are 32-bit (the planner keeps 9 planes below 2^31).
struct Nbr {
    int col[3];
    int row[3];
};

__device__ __forceinline__ void periodic_rows(const SampleDev& sp, int y, Nbr& n) {
    const int ym = y == 0 ? sp.ny - 1 : y - 1, yp = y == sp.ny - 1 ? 0 : y + 1;
    n.row[0] = ym * sp.pitch;
    n.row[1] = y * sp.pitch;
    n.row[2] = yp * sp.pitch;
}
__device__ __forceinline__ void periodic_cols(const SampleDev& sp, int x, Nbr& n) {
    n.col[0] = x == 0 ? sp.nx - 1 : x - 1;
    n.col[1] = x;
    n.col[2] = x == sp.nx - 1 ? 0 : x + 1;
}

// Nine incoming shifted populations of node (x, y) at step t.
// links: Bouzidi obstacle links of the node (bit i), 0 for every other node.
template <typename S, bool ODD>
__device__ __forceinline__ void node_load(const KParams& p, const SampleDev& sp, const S* base,
                                          const uint32_t* mask, int x, int y, int t, bool chan,
                                          const Nbr& nb, const InitDev* bz, uint32_t links,
                                          typename Storage<S>::C (&g)[9], const typename Storage<S>::Q& qz,
                                          bool end_columns = true) {
    using C = typename Storage<S>::C;
    const int plane = (int)sp.plane;
    if (chan && end_columns && sp.inout && t > 0 && (x == 0 || x == sp.nx - 1)) {
        // interpolated inlet/outlet: the end columns' state was formed after the last step
        const double* b = p.bcpop + (int64_t)(sp.bc_off + (x == 0 ? 0 : sp.ny) + y) * 9;
#pragma unroll
        for (int i = 0; i < 9; ++i) g[i] = (C)b[i];
        return;
    }
    if (!ODD) {
        const int own = nb.row[1] + x;
#pragma unroll
        for (int i = 0; i < 9; ++i) g[i] = Storage<S>::load(base + (i * plane + own), qz, i);
        if (chan && links) bouzidi_complete(*bz, x, y, links, g);
    } else if (!chan) {
#pragma unroll
        for (int i = 0; i < 9; ++i)
            g[i] = Storage<S>::load(base + (opp(i) * plane + nb.row[1 - cy(i)] + nb.col[1 - cx(i)]), qz, i);
    } else {
        C ubx = C(0), uby = C(0);
        if (chan && x == sp.nx - 1) {
            if (sizeof(C) == 8) {
                ubx = (C)p.side_d[2 * (sp.side_off + y)];
                uby = (C)p.side_d[2 * (sp.side_off + y) + 1];
            } else {
                ubx = (C)p.side[2 * (sp.side_off + y)];
                uby = (C)p.side[2 * (sp.side_off + y) + 1];
            }
        }
        g[0] = Storage<S>::load(base + (nb.row[1] + x), qz, 0);
#pragma unroll
        for (int i = 1; i < 9; ++i) g[i] = read_incoming<S>(base, sp, mask, x, y, i, t - 1, ubx, uby, chan, qz);
        if (links) bouzidi_complete(*bz, x, y, links, g);
    }
}

// Moments, QoI contributions, BGK and the streaming stores of node (x, y) at step t.
template <typename S, bool ODD>
__device__ __forceinline__ void node_update(const KParams& p, const SampleDev& sp, S* base, const uint32_t* mask,
                                            int x, int y, int t, bool chan, bool want_k, bool want_f,
                                            const Nbr& nb, const InitDev* bz, uint32_t links,
                                            typename Storage<S>::C (&g)[9], double (&red)[3],
                                            const typename Storage<S>::Q& qz) {
    using C = typename Storage<S>::C;
    const int own = nb.row[1] + x;
    const int plane = (int)sp.plane;
    // stochastic-rounding bits: one mixed word per node and step, spread over the nine stores by
    // distinct odd multipliers (the high 16 bits of the products are used)
    const bool sr = sizeof(S) == 2 && p.stochastic != 0;
    const uint32_t h = sr ? mix32((uint32_t)own * 0x9E3779B1u + (uint32_t)t * 0x85EBCA77u +
                                  (uint32_t)sp.sample_id * 0xC2B2AE3Du)
                          : 0u;
    auto put = [&](S* ptr, C v, int i) {
        if (sr)
            Storage<S>::store_sr(ptr, v, (h * (0x2545F491u + 0x6A09E668u * (uint32_t)i)) >> 16, qz, i);
        else
            Storage<S>::store(ptr, v, qz, i);
    };
    C drho, jx, jy, ux, uy;
    moments(g, drho, jx, jy, ux, uy);
    if (want_k) red[0] += (double)(ux * ux + uy * uy);
    if (chan && !ODD && x == sp.nx - 1) {
        if (sizeof(C) == 8) {
            p.side_d[2 * (sp.side_off + y)] = (double)ux;
            p.side_d[2 * (sp.side_off + y) + 1] = (double)uy;
        } else {
            p.side[2 * (sp.side_off + y)] = (float)ux;
            p.side[2 * (sp.side_off + y) + 1] = (float)uy;
        }
    }
    bgk(g, (C)sp.omega, drho, jx, jy, ux, uy);
    if (want_f && mask != nullptr) {
        C fx = C(0), fy = C(0);
#pragma unroll
        for (int i = 1; i < 9; ++i) {
            const int xn = x + cx(i), yn = y + cy(i);
            if (xn >= 0 && xn < sp.nx && yn >= 0 && yn < sp.ny && mask_solid(mask, mask_words(sp), xn, yn)) {
                const C fs = g[i] + wgt<C>(i);
                fx += C(2 * cx(i)) * fs;
                fy += C(2 * cy(i)) * fs;
            }
        }
        red[1] += (double)fx;
        red[2] += (double)fy;
    }
    if (!ODD) {
        if (chan && links) {
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                if (links >> i & 1u) {
                    put(base + (opp(i) * plane + own), bouzidi_local(*bz, x, y, i, g), i);
                    put(base + ((int64_t)i * plane + (int64_t)(y + cy(i)) * sp.pitch + (x + cx(i))), g[i], i);
                } else {
                    put(base + (opp(i) * plane + own), g[i], i);
                }
            }
            return;
        }
#pragma unroll
        for (int i = 0; i < 9; ++i) put(base + (opp(i) * plane + own), g[i], i);
        return;
    }
    if (!chan) {
#pragma unroll
        for (int i = 0; i < 9; ++i)
            put(base + (i * plane + nb.row[1 + cy(i)] + nb.col[1 + cx(i)]), g[i], i);
        return;
    }
    put(base + own, g[0], 0);
#pragma unroll
    for (int i = 1; i < 9; ++i) {
        int dx = x + cx(i), dy = y + cy(i);
        {
            const int cls = classify(sp, mask, dx, dy);
            const int o = opp(i);
            if (cls == kInterior) {
                put(base + i * plane + (int64_t)dy * sp.pitch + dx, g[i], i);
            } else if (cls == kSolid && (links >> i & 1u)) {
                put(base + o * plane + own, bouzidi_local(*bz, x, y, i, g), i);
                put(base + i * plane + (int64_t)dy * sp.pitch + dx, g[i], i);  // parked g*_i
            } else if (cls == kWall || cls == kSolid) {
                put(base + o * plane + own, g[i], i);
            } else if (cls == kInlet) {
                const C yy = C(y) + C(0.5) - C(0.5) * C(cy(o));
                put(base + o * plane + own, g[i] + C(6) * wgt<C>(o) * C(cx(o)) * inflow<C>(sp, yy, t), i);
            } else {
                const C cu = C(cx(o)) * ux + C(cy(o)) * uy;
                put(base + o * plane + own, -g[i] + wgt<C>(o) * (C(9) * cu * cu - C(3) * (ux * ux + uy * uy)), i);
            }
        }
    }
}

// C_D, C_L of sample j at time s (a QoI step) into the series, and the steady-state test: a
// sample whose C_D changed by less than steady_tol |C_D| at steady_checks consecutive checks
// stops with its state at s.
__device__ __forceinline__ void record_force(const KParams& p, const SampleDev& sp, int j, int s, double fx,
                                             double fy) {
    const double cd = fx * sp.force_norm, cl = fy * sp.force_norm;
    const int64_t col = s / p.qoi_every - 1;
    if (p.series) p.series[(int64_t)sp.sample_id * p.series_ld + col] = cd;
    if (p.series_cl) p.series_cl[(int64_t)sp.sample_id * p.series_ld + col] = cl;
    if (sp.steady_tol > 0.0) {
        const double prev = p.cd_prev[sp.slot];
        const bool pass = !isnan(prev) && fabs(cd - prev) < sp.steady_tol * fabs(cd);
        const int run = pass ? p.streak[sp.slot] + 1 : 0;
        p.streak[sp.slot] = run;
        if (run >= sp.steady_checks) {
            p.done[sp.slot] = 1;
            p.steps_run[sp.slot] = s;
            atomicAdd(p.n_done, 1);
        }
        p.cd_prev[sp.slot] = cd;
    }
}

// Shared state of one block while it processes a tile.
template <int NT>
struct TileShared {
    int nact, ntiles, j, flag;
    long long ticket;
    double red[(NT / 32) * 3];
    __align__(16) SampleDev sp;
};

// One tile = (32 NPT) columns x TR rows of one sample; thread (lane, row) owns the NPT nodes
// x = x0 + lane + 32 k, so every warp-wide access of a population plane is contiguous.  All
// NPT x 9 loads of a thread are issued before any arithmetic.
// MIXED: the batch holds channel samples; each tile then branches on its own sample's kind.
template <typename S, bool ODD, bool MIXED, int TR, int NPT>
__device__ __forceinline__ void process_tile(const KParams& p, int t, int tile, int nact, bool k_step, bool f_step,
                                             TileShared<kTileCols * TR>& sh) {
    using C = typename Storage<S>::C;
    constexpr int NT = kTileCols * TR;
    if (threadIdx.y == 0) {  // warp 0 fetches the sample record (32 words) into shared memory
        const int jj = tile_sample(p, tile, nact);
        reinterpret_cast<uint32_t*>(&sh.sp)[threadIdx.x] =
            __ldg(reinterpret_cast<const uint32_t*>(p.samples + jj) + threadIdx.x);
        if (threadIdx.x == 0) sh.j = jj;
    }
    __syncthreads();
    const int j = sh.j;
    const SampleDev& sp = sh.sp;
    const bool chan = MIXED && sp.kind == UQLB_CASE_CHANNEL;
    const typename Storage<S>::Q qz = quanta_of<S>(p, j);
    if (chan && p.done[sp.slot]) {
        __syncthreads();
        return;
    }
    const bool want_k = k_step && !chan;
    const bool want_f = f_step && chan && !sp.bouzidi;  // Bouzidi forces: bouzidi_force_kernel
    const int lt = tile - sp.tile_base;
    const int x0 = (lt % sp.tiles_x) * (kTileCols * NPT) + threadIdx.x;
    const int y = (lt / sp.tiles_x) * TR + threadIdx.y;
    // A channel node at least one node inside the walls and the end columns and outside the
    // obstacle's box (every node that is solid or has a solid neighbour lies in it) has no boundary
    // link: it takes the periodic node path (the same loads, stores and arithmetic, no link
    // classification).  Boundary nodes outside the box classify their links without the mask.  A
    // tile of such inner nodes only skips the box and mask set-up.  The sample-level QoI logic
    // (want_f, the tile reduction) stays on the sample's kind.
    int bb[4] = {0, -1, 0, -1};
    bool inner_tile = !chan;
    if (chan) {
        const InitDev& in = p.init[j];
        for (int q = 0; q < 4; ++q) bb[q] = in.bbox[q];
        const int tx0 = (lt % sp.tiles_x) * (kTileCols * NPT), ty0 = (lt / sp.tiles_x) * TR;
        const int tx1 = tx0 + kTileCols * NPT - 1, ty1 = ty0 + TR - 1;
        inner_tile = tx0 >= 1 && tx1 <= sp.nx - 2 && ty0 >= 1 && ty1 <= sp.ny - 2 &&
                     (tx1 < bb[0] || tx0 > bb[1] || ty1 < bb[2] || ty0 > bb[3]);
    }
    const uint32_t* mask = (!inner_tile && sp.mask_off >= 0) ? p.masks + sp.mask_off : nullptr;
    S* base = static_cast<S*>(p.arena) + sp.f_off;

    const InitDev* bz = (!inner_tile && sp.bouzidi && mask != nullptr) ? p.init + j : nullptr;
    C g[NPT][9];
    bool act[NPT], nc[NPT];
    uint32_t lk[NPT];
    const uint32_t* mk[NPT];
    Nbr nb[NPT];
    Nbr rows;
    if (ODD) {
        periodic_rows(sp, y, rows);
    } else {
        rows.row[1] = y * sp.pitch;
    }
    const bool y_inner = y >= 1 && y <= sp.ny - 2;
#pragma unroll
    for (int k = 0; k < NPT; ++k) {
        const int x = x0 + kTileCols * k;
        const bool in_box = x >= bb[0] && x <= bb[1] && y >= bb[2] && y <= bb[3];
        nc[k] = !inner_tile && !(y_inner && x >= 1 && x <= sp.nx - 2 && !in_box);
        mk[k] = in_box ? mask : nullptr;
        nb[k] = rows;
        if (ODD) periodic_cols(sp, x, nb[k]);
        act[k] = x < sp.nx && y < sp.ny;
        if (act[k] && mk[k] != nullptr) act[k] = !mask_solid(mk[k], mask_words(sp), x, y);
        lk[k] = (act[k] && bz != nullptr && in_box) ? obstacle_links(sp, *bz, mk[k], x, y) : 0u;
        if (act[k]) node_load<S, ODD>(p, sp, base, mk[k], x, y, t, nc[k], nb[k], bz, lk[k], g[k], qz);
    }
    double red[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int k = 0; k < NPT; ++k)
        if (act[k])
            node_update<S, ODD>(p, sp, base, mk[k], x0 + kTileCols * k, y, t, nc[k], want_k, want_f, nb[k], bz, lk[k],
                                g[k], red, qz);

    if (want_k || want_f) {
        double tot[3];
        if (tile_reduce_last<3, NT>(p, sp, j, tile, red, tot, sh.red, &sh.flag)) {
            if (threadIdx.x == 0 && threadIdx.y == 0) {
                if (want_k) {
                    p.series[(int64_t)sp.sample_id * p.series_ld + t / p.qoi_every] = tot[0] * sp.u_ref_inv2;
                } else {
                    record_force(p, sp, j, t + 1, tot[1], tot[2]);
                }
            }
        }
    } else {
        __syncthreads();
    }
}

// Active samples and tiles of step t, published in shared memory by thread 0.
template <int NT>
__device__ __forceinline__ void step_extent(const KParams& p, int t, TileShared<NT>& sh) {
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        const int nact = active_samples(p, t);
        sh.nact = nact;
        sh.ntiles = nact > 0 ? p.samples[nact - 1].tile_base + p.samples[nact - 1].tiles : 0;
    }
    __syncthreads();
}

// One launch per time step: a grid sized to the resident blocks strides over the active tiles.
template <typename S, bool ODD, bool MIXED, int TR, int NPT>
__global__ void __launch_bounds__(kTileCols* TR) step_kernel(KParams p) {
    __shared__ TileShared<kTileCols * TR> sh;
    const int t = (int)(*p.step_counter) + p.dt;
    if (t >= p.max_steps) return;
    step_extent(p, t, sh);
    const int nact = sh.nact, ntiles = sh.ntiles;
    const bool k_step = p.qoi_every > 0 && p.series != nullptr && (t % p.qoi_every) == 0;
    const bool f_step = MIXED && p.qoi_every > 0 && ((t + 1) % p.qoi_every) == 0;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x)
        process_tile<S, ODD, MIXED, TR, NPT>(p, t, tile, nact, k_step, f_step, sh);
}

// Wall-clock nanoseconds of the device.
__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long v;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(v));
    return v;
}

// Grid-wide barrier of a cooperative launch (all blocks resident).  The wait is bounded: after
// kBarrierTimeoutNs without the last arrival the block records UQLB_ERR_TIMEOUT and every block
// returns at its next barrier.  `arrive` = false withholds this block's arrival (test hook that
// makes the other blocks' wait run out).
constexpr unsigned long long kBarrierTimeoutNs = 2000000000ull;

__device__ __forceinline__ bool grid_barrier(const KParams& p, bool arrive) {
    __syncthreads();
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        volatile unsigned int* gen = p.bar_gen;
        const unsigned int g = *gen;
        __threadfence();
        bool waited = true;
        if (arrive && atomicAdd(p.bar_count, 1u) == gridDim.x - 1) {
            atomicExch(p.bar_count, 0u);
            __threadfence();
            atomicAdd(p.bar_gen, 1u);
            waited = false;
        }
        if (waited) {
            const unsigned long long start = globaltimer_ns();
            while (*gen == g && *(volatile int*)p.bar_err == 0) {
                if (globaltimer_ns() - start > kBarrierTimeoutNs) {
                    atomicExch(p.bar_err, UQLB_ERR_TIMEOUT);
                    break;
                }
                __nanosleep(256);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return *(volatile int*)p.bar_err == 0;
}

// Persistent mode: one cooperative launch runs `chunk` time steps.  Tiles are handed out by a
// single ticket counter (the per-tile work queue): step t owns tickets [base_t, base_t + ntiles_t);
// a block that draws a ticket of a later step keeps it across the barrier and processes it there.
template <typename S, bool MIXED, int TR, int NPT>
__global__ void __launch_bounds__(kTileCols* TR) persistent_kernel(KParams p, int chunk) {
    __shared__ TileShared<kTileCols * TR> sh;
    const int t0 = (int)(*p.step_counter);
    long long base = 0, ticket = -1;
    for (int dt = 0; dt < chunk; ++dt) {
        const int t = t0 + dt;
        if (t >= p.max_steps) break;
        step_extent(p, t, sh);
        const int nact = sh.nact, ntiles = sh.ntiles;
        const bool k_step = p.qoi_every > 0 && p.series != nullptr && (t % p.qoi_every) == 0;
        const bool f_step = MIXED && p.qoi_every > 0 && ((t + 1) % p.qoi_every) == 0;
        while (true) {
            if (ticket < 0) {
                if (threadIdx.x == 0 && threadIdx.y == 0) sh.ticket = (long long)atomicAdd(p.tickets, 1ull);
                __syncthreads();
                ticket = sh.ticket;
                __syncthreads();
            }
            if (ticket >= base + ntiles) break;
            const int tile = (int)(ticket - base);
            if (t & 1)
                process_tile<S, true, MIXED, TR, NPT>(p, t, tile, nact, k_step, f_step, sh);
            else
                process_tile<S, false, MIXED, TR, NPT>(p, t, tile, nact, k_step, f_step, sh);
            ticket = -1;
        }
        base += ntiles;
        const bool arrive = !(p.test_withhold && blockIdx.x == 0);
        if (!grid_barrier(p, arrive)) return;
    }
}

// ------------------------------------------------------------------------------------------
// Two-step scheme (periodic batches): one launch moves every running sample two steps ahead,
// from one lattice to the other.  A block loads its tile with a one-node halo (natural layout,
// periodic wrap), collides it into shared memory, then streams from shared memory, collides the
// tile again and pushes the result into the other lattice.  HBM traffic per launch: the tile and
// its halo read once, the tile written once.  A sample with one step left takes one
// collide-and-push step.  Every launch of a run moves each running sample to the other lattice,
// so at the launch of step t (t - t0 even, t0 the run's first step) a sample's state is on
// lattice sel ^ ((t - t0) / 2 & 1).
// ------------------------------------------------------------------------------------------
// Launches of a run started at step t0 that a sample ending at step t_end takes part in (spl steps
// per launch; a sample's last launch may run fewer).
__device__ __forceinline__ int launches_of(int t_end, int t0, int spl) {
    return t_end > t0 ? (t_end - t0 + spl - 1) / spl : 0;
}

__device__ __forceinline__ bool on_final_second(const KParams& p, int slot, int T) {
    return ((p.sel[slot] ^ launches_of(T, (int)p.step_counter[1], p.spl)) & 1) != 0;
}

// Tuning of the two-step kernel (measured on the 625 x 256^2 FP32 ensemble): nodes per load
// batch of the halo phase, resident blocks per SM requested for 8-row tiles (register budget
// 65536 / (256 x blocks); 4-row tiles get twice as many), and packed FP32 arithmetic.
#ifndef UQLB_STEP2_BATCH
#define UQLB_STEP2_BATCH 2
#endif
#ifndef UQLB_STEP2_BLOCKS8
#define UQLB_STEP2_BLOCKS8 4
#endif
#ifndef UQLB_STEP2_PACKED
#define UQLB_STEP2_PACKED 1
#endif

// BGK collision of one node in place; adds u.u to acc when want.
template <typename C>
__device__ __forceinline__ void collide_one(C (&g)[9], C omega, bool want, double& acc) {
    C drho, jx, jy, ux, uy;
    moments(g, drho, jx, jy, ux, uy);
    if (want) acc += (double)(ux * ux + uy * uy);
    bgk(g, omega, drho, jx, jy, ux, uy);
}

// Shared-memory tile [9][eh][ew]: store one node's populations / gather the populations that
// stream into node (ey, ex) (population i comes from (ey - c_iy, ex - c_ix)).
template <typename C>
__device__ __forceinline__ void tile_store(C* sm, int eh, int ew, int ey, int ex, const C (&g)[9]) {
#pragma unroll
    for (int i = 0; i < 9; ++i) sm[(i * eh + ey) * ew + ex] = g[i];
}
template <typename C>
__device__ __forceinline__ void tile_gather(const C* sm, int eh, int ew, int ey, int ex, C (&g)[9]) {
#pragma unroll
    for (int i = 0; i < 9; ++i) g[i] = sm[(i * eh + ey - cy(i)) * ew + ex - cx(i)];
}

template <typename S, int TR, int NPT>
__global__ void __launch_bounds__(kTileCols* TR, TR == 4 ? 2 * UQLB_STEP2_BLOCKS8 : (TR == 8 ? UQLB_STEP2_BLOCKS8 : 1))
    step2_kernel(KParams p) {
    using C = typename Storage<S>::C;
    constexpr int NT = kTileCols * TR, TW = kTileCols * NPT, EW = TW + 2, EH = TR + 2;
    __shared__ TileShared<NT> sh;
    extern __shared__ __align__(16) unsigned char s2_raw[];
    C* sm = reinterpret_cast<C*>(s2_raw);  // post-collision tile + halo, [9][EH][EW]
    const int t = (int)p.step_counter[0] + p.dt;
    const int t0 = (int)p.step_counter[1];
    step_extent(p, t, sh);
    const int nact = sh.nact, ntiles = sh.ntiles;
    const bool want_a = p.qoi_every > 0 && p.series != nullptr && (t % p.qoi_every) == 0;
    const bool want_b0 = p.qoi_every > 0 && p.series != nullptr && ((t + 1) % p.qoi_every) == 0;
    const int lane = threadIdx.x, ty = threadIdx.y;
    const bool sr = sizeof(S) == 2 && p.stochastic != 0;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        if (ty == 0) {
            const int jj = tile_sample(p, tile, nact);
            reinterpret_cast<uint32_t*>(&sh.sp)[lane] = __ldg(reinterpret_cast<const uint32_t*>(p.samples + jj) + lane);
            if (lane == 0) sh.j = jj;
        }
        __syncthreads();
        const int j = sh.j;
        const SampleDev& sp = sh.sp;
        const typename Storage<S>::Q qz = quanta_of<S>(p, j);
        const bool two = t + 1 < sp.steps;
        const bool want_b = two && want_b0;
        const int lt = tile - sp.tile_base;
        const int x0 = (lt % sp.tiles_x) * TW, y0 = (lt / sp.tiles_x) * TR;
        const int wa = min(TW, sp.nx - x0), ha = min(TR, sp.ny - y0);  // active columns and rows
        const bool second = ((p.sel[sp.slot] ^ ((t - t0) >> 1)) & 1) != 0;
        const S* src = static_cast<const S*>(second ? p.arena2 : p.arena) + sp.f_off;
        S* dst = static_cast<S*>(second ? p.arena : p.arena2) + sp.f_off;
        const int plane = (int)sp.plane, pitch = sp.pitch, nx = sp.nx, ny = sp.ny;
        const C omega = (C)sp.omega;
        const PackedBGK omega2 = packed_bgk((float)omega);
        double red[2] = {0.0, 0.0};
        // collide-and-push of one node's post-collision populations g (step ts) into dst
        auto push = [&](int x, int y, int ts, const C (&g)[9]) {
            const int xm = x == 0 ? nx - 1 : x - 1, xp = x == nx - 1 ? 0 : x + 1;
            const int ym = y == 0 ? ny - 1 : y - 1, yp = y == ny - 1 ? 0 : y + 1;
            const int col[3] = {xm, x, xp};
            const int row[3] = {ym * pitch, y * pitch, yp * pitch};
            const uint32_t h = sr ? mix32((uint32_t)(y * pitch + x) * 0x9E3779B1u + (uint32_t)ts * 0x85EBCA77u +
                                          (uint32_t)sp.sample_id * 0xC2B2AE3Du)
                                  : 0u;
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                S* ptr = dst + (i * plane + row[1 + cy(i)] + col[1 + cx(i)]);
                if (sr)
                    Storage<S>::store_sr(ptr, g[i], (h * (0x2545F491u + 0x6A09E668u * (uint32_t)i)) >> 16, qz, i);
                else
                    Storage<S>::store(ptr, g[i], qz, i);
            }
        };
        if (!two) {
            const int y = y0 + ty;
            C g[NPT][9];
#pragma unroll
            for (int k = 0; k < NPT; ++k) {
                const int x = x0 + lane + kTileCols * k;
                if (lane + kTileCols * k < wa && ty < ha) {
#pragma unroll
                    for (int i = 0; i < 9; ++i) g[k][i] = Storage<S>::load(src + (i * plane + y * pitch + x), qz, i);
                }
            }
#pragma unroll
            for (int k = 0; k < NPT; ++k) {
                const int x = x0 + lane + kTileCols * k;
                if (lane + kTileCols * k < wa && ty < ha) {
                    C drho, jx, jy, ux, uy;
                    moments(g[k], drho, jx, jy, ux, uy);
                    if (want_a) red[0] += (double)(ux * ux + uy * uy);
                    bgk(g[k], omega, drho, jx, jy, ux, uy);
                    push(x, y, t, g[k]);
                }
            }
        } else {
            // phase A: the tile and its halo at step t, post-collision values into shared memory.
            // The (TW + 2) x (TR + 2) nodes are dealt out row-major over all threads, MB at a
            // time (all their loads issued before any arithmetic).
            constexpr int EXT = EW * EH, MB = sizeof(C) == 4 ? UQLB_STEP2_BATCH : 3;
            const int tid = lane + kTileCols * ty;
#pragma unroll 1
            for (int e0 = 0; e0 < EXT; e0 += NT * MB) {
                C g[MB][9];
                int ex[MB], ey[MB];
                bool ok[MB];
#pragma unroll
                for (int m = 0; m < MB; ++m) {
                    const int e = e0 + tid + NT * m;
                    ey[m] = e / EW;
                    ex[m] = e - ey[m] * EW;
                    ok[m] = e < EXT && ex[m] <= wa + 1 && ey[m] <= ha + 1;
                    if (ok[m]) {
                        int gx = x0 - 1 + ex[m], gy = y0 - 1 + ey[m];
                        gx = gx < 0 ? gx + nx : (gx >= nx ? gx - nx : gx);
                        gy = gy < 0 ? gy + ny : (gy >= ny ? gy - ny : gy);
                        const S* q = src + (gy * pitch + gx);
#pragma unroll
                        for (int i = 0; i < 9; ++i) g[m][i] = Storage<S>::load(q + i * plane, qz, i);
                    }
                }
                if constexpr (UQLB_STEP2_PACKED && sizeof(C) == 4 && MB % 2 == 0) {
                    // two nodes per packed collision where both are present
#pragma unroll
                    for (int pr = 0; pr < MB / 2; ++pr) {
                        const int m0 = 2 * pr, m1 = 2 * pr + 1;
                        const bool in0 = ex[m0] >= 1 && ex[m0] <= wa && ey[m0] >= 1 && ey[m0] <= ha;
                        const bool in1 = ex[m1] >= 1 && ex[m1] <= wa && ey[m1] >= 1 && ey[m1] <= ha;
                        if (ok[m0] && ok[m1]) {
                            float qa = 0.0f, qb = 0.0f;
                            collide_pair(g[m0], g[m1], omega2, want_a ? &qa : nullptr, want_a ? &qb : nullptr);
                            if (want_a && in0) red[0] += (double)qa;
                            if (want_a && in1) red[0] += (double)qb;
                            tile_store(sm, EH, EW, ey[m0], ex[m0], g[m0]);
                            tile_store(sm, EH, EW, ey[m1], ex[m1], g[m1]);
                        } else {
                            if (ok[m0]) {
                                collide_one(g[m0], omega, want_a && in0, red[0]);
                                tile_store(sm, EH, EW, ey[m0], ex[m0], g[m0]);
                            }
                            if (ok[m1]) {
                                collide_one(g[m1], omega, want_a && in1, red[0]);
                                tile_store(sm, EH, EW, ey[m1], ex[m1], g[m1]);
                            }
                        }
                    }
                } else {
#pragma unroll
                    for (int m = 0; m < MB; ++m) {
                        if (!ok[m]) continue;
                        const bool in = ex[m] >= 1 && ex[m] <= wa && ey[m] >= 1 && ey[m] <= ha;
                        collide_one(g[m], omega, want_a && in, red[0]);
                        tile_store(sm, EH, EW, ey[m], ex[m], g[m]);
                    }
                }
            }
            __syncthreads();
            // phase B: stream from shared memory, collide at step t + 1, push into the other lattice
            const int y = y0 + ty, ey = ty + 1;
            if (ty < ha) {
                if constexpr (UQLB_STEP2_PACKED && sizeof(C) == 4 && NPT % 2 == 0) {
#pragma unroll
                    for (int pr = 0; pr < NPT / 2; ++pr) {
                        const int ea = lane + kTileCols * (2 * pr) + 1, eb = ea + kTileCols;
                        if (eb <= wa) {
                            C ga[9], gb[9];
                            tile_gather(sm, EH, EW, ey, ea, ga);
                            tile_gather(sm, EH, EW, ey, eb, gb);
                            float qa = 0.0f, qb = 0.0f;
                            collide_pair(ga, gb, omega2, want_b ? &qa : nullptr, want_b ? &qb : nullptr);
                            if (want_b) {
                                red[1] += (double)qa;
                                red[1] += (double)qb;
                            }
                            push(x0 + ea - 1, y, t + 1, ga);
                            push(x0 + eb - 1, y, t + 1, gb);
                        } else if (ea <= wa) {
                            C ga[9];
                            tile_gather(sm, EH, EW, ey, ea, ga);
                            collide_one(ga, omega, want_b, red[1]);
                            push(x0 + ea - 1, y, t + 1, ga);
                        }
                    }
                } else {
#pragma unroll
                    for (int k = 0; k < NPT; ++k) {
                        const int ex = lane + kTileCols * k + 1;
                        if (ex > wa) continue;
                        C g[9];
                        tile_gather(sm, EH, EW, ey, ex, g);
                        collide_one(g, omega, want_b, red[1]);
                        push(x0 + ex - 1, y, t + 1, g);
                    }
                }
            }
        }
        if (want_a || want_b) {
            double tot[2];
            if (tile_reduce_last<2, NT>(p, sp, j, tile, red, tot, sh.red, &sh.flag)) {
                if (lane == 0 && ty == 0) {
                    if (want_a) p.series[(int64_t)sp.sample_id * p.series_ld + t / p.qoi_every] = tot[0] * sp.u_ref_inv2;
                    if (want_b)
                        p.series[(int64_t)sp.sample_id * p.series_ld + (t + 1) / p.qoi_every] = tot[1] * sp.u_ref_inv2;
                }
            }
        } else {
            __syncthreads();  // the next tile reuses shared memory
        }
    }
}

// ------------------------------------------------------------------------------------------
// Two steps per launch by row strips (periodic batches of one width nx, a multiple of 64).
// ------------------------------------------------------------------------------------------
// The rows of the running samples, taken sample after sample in table order, are split into
// gridDim.x ranges of equal length; a block of nx / 2 threads walks its range row by row, thread
// k owning the node pair (2k, 2k + 1) of every row.  For row y of a sample it collides row y + 1
// at step t into a ring in shared memory (phase A), waits at one barrier, then gathers row y's
// populations of step t + 1 from rows y - 1, y and y + 1 of the ring, collides them and pushes
// them into the other lattice (phase B).  Phase A visits every row once plus two rows before the
// first row of each (range, sample) piece, against (TR + 2)(TW + 2) / (TR TW) nodes per tile
// node in step2_kernel, and the loop keeps each thread's columns, so no per-node index
// arithmetic or wrap-around remains apart from the two edge columns.
//
// Ring: population i of a phase-A row is read by the phase-B row y + c_iy, so the group with
// c_iy = +1 (i = 2, 5, 6) lives two iterations, c_iy = 0 (0, 1, 3) one and c_iy = -1 (4, 7, 8)
// none; with one barrier per row the next phase-A row may be written while a slower thread is
// still gathering, which takes one more slot each: 4, 3 and 2 slots of 3 planes of nx floats.
constexpr int kStripPlanes = 27;
// FP32 rows are staged one row ahead by asynchronous copies; with a 196 KB share of shared memory
// per SM (5 blocks at nx = 256) the L1 keeps 60 KB for the copies in flight, where the largest
// share leaves 28 KB and caps the bytes in flight (141 against 178 GLUPS on the 625 x 256^2
// ensemble).  16-bit rows have half the bytes in flight and gain more from warps: no staging, the
// largest share (8 blocks).
#ifndef UQLB_STRIP_PREFETCH_F32
#define UQLB_STRIP_PREFETCH_F32 1
#endif
#ifndef UQLB_STRIP_PREFETCH_16
#define UQLB_STRIP_PREFETCH_16 0
#endif
#ifndef UQLB_STRIP_CARVEOUT_F32_KB
#define UQLB_STRIP_CARVEOUT_F32_KB 196
#endif
#ifndef UQLB_STRIP_CARVEOUT_16_KB
#define UQLB_STRIP_CARVEOUT_16_KB 0
#endif
template <typename S>
struct StripTune {
    static constexpr int depth = sizeof(S) == 4 ? UQLB_STRIP_PREFETCH_F32 : UQLB_STRIP_PREFETCH_16;  // staged rows
    static constexpr int carveout_kb = sizeof(S) == 4 ? UQLB_STRIP_CARVEOUT_F32_KB : UQLB_STRIP_CARVEOUT_16_KB;
    // widest rows whose ring and staging fit one block's 227 KB (less 2 KB of static and reserve)
    static constexpr int max_nx_raw = (232448 - 2048) / (kStripPlanes * 4 + depth * 9 * (int)sizeof(S)) / 64 * 64;
    static constexpr int max_nx = max_nx_raw < 2048 ? max_nx_raw : 2048;
};
// Threads of a block for rows of width nx: one per node pair, whole warps; the ring is twice as wide.
inline int strip_threads(int nx) { return ((nx + 1) / 2 + 31) / 32 * 32; }

// Asynchronous copy of N bytes (4 or 8) from global to shared memory.  Each thread commits one
// group per staged row and waits with cp_async_wait<D - 1>() until its own oldest group has landed
// (a thread reads back only what it copied itself, so no barrier is needed for the staging).
template <int N>
__device__ __forceinline__ void cp_async(void* smem, const void* gmem) {
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(a), "l"(gmem), "n"(N) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Slot plane of direction i for the phase-A row with sequence number q (q = row - first + 1).
__device__ __forceinline__ int strip_plane(int i, int q) {
    switch (i) {
        case 2: return (q & 3) * 3 + 0;
        case 5: return (q & 3) * 3 + 1;
        case 6: return (q & 3) * 3 + 2;
        case 0: return 12 + (q % 3) * 3 + 0;
        case 1: return 12 + (q % 3) * 3 + 1;
        case 3: return 12 + (q % 3) * 3 + 2;
        case 4: return 21 + (q & 1) * 3 + 0;
        case 7: return 21 + (q & 1) * 3 + 1;
        default: return 21 + (q & 1) * 3 + 2;
    }
}

// Two adjacent populations i (an even column and the next) as one packed pair: the pair's stored
// values as one register (PairRaw: two 16-bit values in a word, or two FP32 values) and their
// conversion (pair_from_raw); pair_load reads the register from memory.
template <typename S>
struct PairRawT {
    using T = uint32_t;
};
template <>
struct PairRawT<float> {
    using T = f2;
};
template <typename S>
using PairRaw = typename PairRawT<S>::T;
template <typename S>
__device__ __forceinline__ f2 pair_from_raw(PairRaw<S> w, const typename Storage<S>::Q& qz, int i);
template <>
__device__ __forceinline__ f2 pair_from_raw<float>(f2 w, const NoQuanta&, int) {
    return w;
}
template <>
__device__ __forceinline__ f2 pair_from_raw<__half>(uint32_t w, const NoQuanta&, int) {
    const float2 v = __half22float2(*reinterpret_cast<const __half2*>(&w));
    return pk(v.x * 0x1p-12f, v.y * 0x1p-12f);
}
template <>
__device__ __forceinline__ f2 pair_from_raw<__nv_bfloat16>(uint32_t w, const NoQuanta&, int) {
    const float2 v = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&w));
    return pk(v.x, v.y);
}
template <>
__device__ __forceinline__ f2 pair_from_raw<int16_t>(uint32_t w, const Quanta& qz, int i) {
    // each signed value plus 2^15 becomes the low mantissa bits of 2^23 (byte permutes, no integer
    // conversion); one packed subtraction of 2^23 + 2^15 gives the two integers exactly and one
    // packed multiply scales them: the same single rounding as (float)q * d
    w ^= 0x80008000u;
    const f2 biased = pk(__uint_as_float(__byte_perm(w, 0x4B000000u, 0x7610)),
                         __uint_as_float(__byte_perm(w, 0x4B000000u, 0x7632)));
    return mul2(sub2(biased, splat(8421376.0f)), splat(qz.d[qclass(i)]));
}
template <typename S>
__device__ __forceinline__ f2 pair_load(const S* ptr, const typename Storage<S>::Q& qz, int i) {
    return pair_from_raw<S>(*reinterpret_cast<const PairRaw<S>*>(ptr), qz, i);
}
// Round-to-nearest store of a pair (each half rounded as Storage<S>::store does).
template <typename S>
__device__ __forceinline__ void pair_store(S* ptr, f2 v, const typename Storage<S>::Q& qz, int i);
template <>
__device__ __forceinline__ void pair_store<float>(float* ptr, f2 v, const NoQuanta&, int) {
    *reinterpret_cast<f2*>(ptr) = v;
}
template <>
__device__ __forceinline__ void pair_store<__half>(__half* ptr, f2 v, const NoQuanta&, int) {
    float a, b;
    upk(v, a, b);
    *reinterpret_cast<__half2*>(ptr) = __floats2half2_rn(a * 0x1p12f, b * 0x1p12f);
}
template <>
__device__ __forceinline__ void pair_store<__nv_bfloat16>(__nv_bfloat16* ptr, f2 v, const NoQuanta&, int) {
    float a, b;
    upk(v, a, b);
    *reinterpret_cast<__nv_bfloat162*>(ptr) = __floats2bfloat162_rn(a, b);
}
template <>
__device__ __forceinline__ void pair_store<int16_t>(int16_t* ptr, f2 v, const Quanta& qz, int i) {
    float a, b;
    upk(v, a, b);
    const uint32_t lo = (uint16_t)Storage<int16_t>::round_nearest(a, qz, i);
    const uint32_t hi = (uint16_t)Storage<int16_t>::round_nearest(b, qz, i);
    *reinterpret_cast<uint32_t*>(ptr) = lo | (hi << 16);
}

// A pair's two 16-bit values as one word (the lower column in bits 15:0), rounded to nearest
// (pair_word) or stochastically (pair_word_sr) with the random bits r: r[15:0] for the lower column,
// r[31:16] for the upper.  The floating formats use cvt.rs, which adds the random bits below the
// kept mantissa and truncates (with FP32 operands scaled as Storage<S>::store scales them); the
// fixed-point format adds them as a fraction of its quantum and rounds down (Storage<int16_t>).
template <typename S>
__device__ __forceinline__ uint32_t pair_word(f2 v, const typename Storage<S>::Q& qz, int i);
template <typename S>
__device__ __forceinline__ uint32_t pair_word_sr(f2 v, uint32_t r, const typename Storage<S>::Q& qz, int i);
template <>
__device__ __forceinline__ uint32_t pair_word<__nv_bfloat16>(f2 v, const NoQuanta&, int) {
    float a, b;
    upk(v, a, b);
    uint32_t d;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(b), "f"(a));
    return d;
}
template <>
__device__ __forceinline__ uint32_t pair_word_sr<__nv_bfloat16>(f2 v, uint32_t r, const NoQuanta&, int) {
    float a, b;
    upk(v, a, b);
    uint32_t d;
    asm("cvt.rs.satfinite.bf16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(b), "f"(a), "r"(r));
    return d;
}
template <>
__device__ __forceinline__ uint32_t pair_word<__half>(f2 v, const NoQuanta&, int) {
    float a, b;
    upk(mul2(v, splat(0x1p12f)), a, b);
    uint32_t d;
    asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(b), "f"(a));
    return d;
}
template <>
__device__ __forceinline__ uint32_t pair_word_sr<__half>(f2 v, uint32_t r, const NoQuanta&, int) {
    float a, b;
    upk(mul2(v, splat(0x1p12f)), a, b);
    uint32_t d;
    asm("cvt.rs.satfinite.f16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(b), "f"(a), "r"(r));
    return d;
}
template <>
__device__ __forceinline__ uint32_t pair_word<int16_t>(f2 v, const Quanta& qz, int i) {
    float a, b;
    upk(v, a, b);
    const uint32_t lo = (uint16_t)Storage<int16_t>::round_nearest(a, qz, i);
    const uint32_t hi = (uint16_t)Storage<int16_t>::round_nearest(b, qz, i);
    return lo | (hi << 16);
}
template <>
__device__ __forceinline__ uint32_t pair_word_sr<int16_t>(f2 v, uint32_t r, const Quanta& qz, int i) {
    float a, b;
    upk(v, a, b);
    const uint32_t lo = (uint16_t)Storage<int16_t>::round_stochastic(a, r, qz, i);
    const uint32_t hi = (uint16_t)Storage<int16_t>::round_stochastic(b, r >> 16, qz, i);
    return lo | (hi << 16);
}

// Random bits of population i of a node pair from the pair's hash h (an odd multiplier per
// population: each maps the uniform h one to one onto 32 bits).
__device__ __forceinline__ uint32_t sr_bits(uint32_t h, int i) { return h * (0x2545F491u + 0x6A09E668u * (uint32_t)i); }

// Block-wide deterministic sum of NV doubles for any whole number of warps; result in thread 0.
template <int NV>
__device__ __forceinline__ void block_sum_dyn(double (&v)[NV], double* smem) {
    const int tid = threadIdx.x, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
    }
    if ((tid & 31) == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) smem[(tid >> 5) * NV + k] = v[k];
    }
    __syncthreads();
    if (tid == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double s = 0.0;
            for (int w = 0; w < nw; ++w) s += smem[w * NV + k];
            v[k] = s;
        }
    }
    __syncthreads();
}

// GENERIC: rows whose width is not the block's 2 x threads (an odd width, or threads past the row);
// rows that fill the block take the unmasked instantiation.
template <typename S, bool GENERIC>
__global__ void __launch_bounds__(1024, 1) strip2_kernel(KParams p) {
    extern __shared__ __align__(16) unsigned char s3_raw[];
    float* ring = reinterpret_cast<float*>(s3_raw);  // [kStripPlanes][nx]
    __shared__ __align__(16) SampleDev s_sp;
    double* s_red = reinterpret_cast<double*>(s3_raw);  // block sums: the ring, once a piece's gathers are done
    __shared__ int s_j, s_rows, s_nact, s_flag;
    const int tid = threadIdx.x, np = blockDim.x;
    const int rw = 2 * np;  // columns of a ring plane: the block's pairs (>= nx)
    // staging slots of the next phase-A row: this thread's pair of each population, [D][9][rw]
    S* stage = reinterpret_cast<S*>(ring + kStripPlanes * rw);
    const int t = (int)p.step_counter[0] + p.dt;
    const int t0 = (int)p.step_counter[1];
    if (tid == 0) {
        const int nact = active_samples(p, t);
        s_nact = nact;
        s_rows = p.row_base[nact];
    }
    __syncthreads();
    const int nact = s_nact, rows = s_rows;
    const int per = (rows + gridDim.x - 1) / gridDim.x;
    const int r0 = blockIdx.x * per, r1 = min(rows, r0 + per);
    const bool want_a = p.qoi_every > 0 && p.series != nullptr && (t % p.qoi_every) == 0;
    const bool want_b0 = p.qoi_every > 0 && p.series != nullptr && ((t + 1) % p.qoi_every) == 0;
    const bool sr = sizeof(S) == 2 && p.stochastic != 0;
    // every sample of a strip batch has the same width: the pair's nodes (a row of odd width ends
    // on a lone node a, whose partner b is read from the row's padding and dropped) and their
    // wrapped neighbour columns
    const int nx = GENERIC ? __ldg(&p.samples[0].nx) : rw;
    const int x = 2 * tid;  // node a; node b is x + 1
    const bool va = !GENERIC || x < nx, vb = !GENERIC || x + 1 < nx;
    const int xl = x == 0 ? nx - 1 : x - 1;                                 // left of a
    const int xar = GENERIC && x + 1 >= nx ? x + 1 - nx : x + 1;            // right of a
    const int xbr = x + 2 >= nx ? x + 2 - nx : x + 2;                       // right of b
    for (int r = r0; r < r1;) {
        __syncthreads();  // the previous piece's gathers are done before the ring is reused
        if (tid == 0) {
            int lo = 0, hi = nact - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (p.row_base[mid] <= r)
                    lo = mid;
                else
                    hi = mid - 1;
            }
            s_j = lo;
        }
        __syncthreads();
        const int j = s_j;
        if (tid < 32) reinterpret_cast<uint32_t*>(&s_sp)[tid] = __ldg(reinterpret_cast<const uint32_t*>(p.samples + j) + tid);
        __syncthreads();
        const int rb = p.row_base[j];
        const int ny = s_sp.ny, pitch = s_sp.pitch, plane = (int)s_sp.plane;
        const int ya = r - rb, yb = min(ny, r1 - rb);
        r = rb + yb;
        const bool two = t + 1 < s_sp.steps;
        const bool want_b = two && want_b0;
        const bool second = ((p.sel[s_sp.slot] ^ ((t - t0) >> 1)) & 1) != 0;
        const S* src = static_cast<const S*>(second ? p.arena2 : p.arena) + s_sp.f_off;
        S* dst = static_cast<S*>(second ? p.arena : p.arena2) + s_sp.f_off;
        const float omega = (float)s_sp.omega;
        const PackedBGK omega2 = packed_bgk(omega);
        const uint32_t sid = (uint32_t)s_sp.sample_id;
        const typename Storage<S>::Q qz = quanta_of<S>(p, j);
        double red[2] = {0.0, 0.0};
        // push of the pair's post-collision populations g (step ts, row y) into dst
        auto push = [&](int y, int ts, const f2 (&g)[9]) {
            const int ym = y == 0 ? ny - 1 : y - 1, yp = y == ny - 1 ? 0 : y + 1;
            const int row[3] = {ym * pitch, y * pitch, yp * pitch};
            uint32_t ha = 0u, hb = 0u;
            if (sr) {
                const uint32_t base = (uint32_t)ts * 0x85EBCA77u + sid * 0xC2B2AE3Du;
                ha = mix32((uint32_t)(y * pitch + x) * 0x9E3779B1u + base);
                hb = mix32((uint32_t)(y * pitch + x + 1) * 0x9E3779B1u + base);
            }
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                S* d = dst + (i * plane + row[1 + cy(i)]);
                float a, b;
                upk(g[i], a, b);
                const int ca = cx(i) == 0 ? x : (cx(i) > 0 ? xar : xl);
                const int cb = cx(i) == 0 ? x + 1 : (cx(i) > 0 ? xbr : x);
                if (sr) {
                    const uint32_t m = 0x2545F491u + 0x6A09E668u * (uint32_t)i;
                    Storage<S>::store_sr(d + ca, a, (ha * m) >> 16, qz, i);
                    if (vb) Storage<S>::store_sr(d + cb, b, (hb * m) >> 16, qz, i);
                } else if (cx(i) == 0 && vb) {
                    pair_store<S>(d + x, g[i], qz, i);
                } else {
                    Storage<S>::store(d + ca, a, qz, i);
                    if (vb) Storage<S>::store(d + cb, b, qz, i);
                }
            }
        };
        auto add_usq = [&](double& acc, f2 q) {
            float a, b;
            upk(q, a, b);
            acc += (double)a;
            if (vb) acc += (double)b;
        };
        if (!two) {
            // the sample's last step: collide and push row by row
            for (int y = ya; y < yb && va; ++y) {
                const S* s0 = src + (y * pitch + x);
                f2 g[9];
#pragma unroll
                for (int i = 0; i < 9; ++i) g[i] = pair_load<S>(s0 + i * plane, qz, i);
                f2 q;
                collide_packed(g, omega2, want_a ? &q : nullptr);
                if (want_a) add_usq(red[0], q);
                push(y, t, g);
            }
        } else {
            // phase A of the row with sequence number q (row ya - 1 + q, periodic)
            auto row_of = [&](int q) {
                const int y = ya - 1 + q;
                return y < 0 ? y + ny : (y >= ny ? y - ny : y);
            };
            // staging: row q of the piece goes to buffer q % D, D rows ahead of its phase A; one copy
            // group per row (empty past the piece), so D - 1 newer groups may stay pending
            constexpr int D = StripTune<S>::depth;
            auto fetch = [&](int q) {
                if (va && q <= yb - ya + 1) {
                    const S* s0 = src + (row_of(q) * pitch + x);
                    S* st = stage + (q % (D > 0 ? D : 1)) * 9 * rw + x;
#pragma unroll
                    for (int i = 0; i < 9; ++i) cp_async<2 * sizeof(S)>(st + i * rw, s0 + i * plane);
                }
                cp_async_commit();
            };
            (void)fetch;
            auto phase_a = [&](int q, bool count) {
                if (!va) return;  // past the row: no node (the barriers are outside)
                f2 g[9];
                if constexpr (D > 0) {
                    cp_async_wait<D - 1>();
                    const S* st = stage + (q % D) * 9 * rw + x;
#pragma unroll
                    for (int i = 0; i < 9; ++i) g[i] = pair_load<S>(st + i * rw, qz, i);
                    fetch(q + D);
                } else {
                    const S* s0 = src + (row_of(q) * pitch + x);
#pragma unroll
                    for (int i = 0; i < 9; ++i) g[i] = pair_load<S>(s0 + i * plane, qz, i);
                }
                f2 qq;
                const bool w = want_a && count;
                collide_packed(g, omega2, w ? &qq : nullptr);
                if (w) add_usq(red[0], qq);
                f2* ring2 = reinterpret_cast<f2*>(ring);
#pragma unroll
                for (int i = 0; i < 9; ++i) ring2[strip_plane(i, q) * np + tid] = g[i];
            };
#pragma unroll
            for (int k = 0; k < D; ++k) fetch(k);
            phase_a(0, false);
            phase_a(1, true);
            for (int y = ya; y < yb; ++y) {
                const int q = y - ya + 1;
                phase_a(q + 1, y + 1 < yb);
                __syncthreads();
                if (!va) continue;
                // phase B: gather row y at step t + 1 (population i from row y - c_iy, column x - c_ix)
                const float* rp = ring + ((q - 1) & 3) * 3 * rw;          // c_iy = +1: row y - 1
                const float* rz = ring + (12 + (q % 3) * 3) * rw;         // c_iy =  0: row y
                const float* rm = ring + (21 + ((q + 1) & 1) * 3) * rw;   // c_iy = -1: row y + 1
                f2 g[9];
                g[0] = *reinterpret_cast<const f2*>(rz + x);
                g[1] = pk(rz[rw + xl], rz[rw + x]);
                g[3] = pk(rz[2 * rw + xar], rz[2 * rw + xbr]);
                g[2] = *reinterpret_cast<const f2*>(rp + x);
                g[5] = pk(rp[rw + xl], rp[rw + x]);
                g[6] = pk(rp[2 * rw + xar], rp[2 * rw + xbr]);
                g[4] = *reinterpret_cast<const f2*>(rm + x);
                g[7] = pk(rm[rw + xar], rm[rw + xbr]);
                g[8] = pk(rm[2 * rw + xl], rm[2 * rw + x]);
                f2 qq;
                collide_packed(g, omega2, want_b ? &qq : nullptr);
                if (want_b) add_usq(red[1], qq);
                push(y, t + 1, g);
            }
        }
        if (want_a || want_b) {
            // this piece's sums; the block that completes the sample adds the pieces in row order
            __syncthreads();  // s_red lives in the ring
            block_sum_dyn<2>(red, s_red);
            if (tid == 0) {
                p.partials[(int64_t)(rb + ya) * 2 + 0] = red[0];
                p.partials[(int64_t)(rb + ya) * 2 + 1] = red[1];
                __threadfence();
                const int prev = atomicAdd(p.counters + j, yb - ya);
                s_flag = (prev + (yb - ya) == ny);
            }
            __syncthreads();
            if (s_flag) {
                __threadfence();
                double acc[2] = {0.0, 0.0};
                for (int q = tid; q < ny; q += np) {
                    if (q == 0 || (rb + q) % per == 0) {
                        acc[0] += __ldcg(p.partials + (int64_t)(rb + q) * 2 + 0);
                        acc[1] += __ldcg(p.partials + (int64_t)(rb + q) * 2 + 1);
                    }
                }
                block_sum_dyn<2>(acc, s_red);
                if (tid == 0) {
                    const int64_t row = (int64_t)s_sp.sample_id * p.series_ld;
                    if (want_a) p.series[row + t / p.qoi_every] = acc[0] * s_sp.u_ref_inv2;
                    if (want_b) p.series[row + (t + 1) / p.qoi_every] = acc[1] * s_sp.u_ref_inv2;
                    p.counters[j] = 0;
                }
            }
        }
    }
}

// ------------------------------------------------------------------------------------------
// Three steps per launch by row strips (periodic batches of one width).
// ------------------------------------------------------------------------------------------
// The same walk as strip2_kernel with one more collision per node: for row y of its range a block
// collides row y + 2 at step t into ring 1 (phase A), waits, gathers row y + 1 of step t + 1 from
// rows y .. y + 2 of ring 1, collides it into ring 2 (phase B), waits, then gathers row y of step
// t + 2 from rows y - 1 .. y + 1 of ring 2, collides it and pushes it into the other lattice
// (phase C).  Each piece (the rows of one sample in one block's range) starts with four extra
// phase-A rows and two extra phase-B rows, so a launch collides (3L + 6) / 3L nodes per node of an
// L-row piece and moves every population through HBM once per three steps (24 B per FP32 node
// update against 36 B with two steps per launch).  A sample with fewer than three steps left runs
// two (phases A and B, B pushing) or one (collide and push) in its last launch.
//
// Rings: population i of a row is read by the next phase at row y + c_iy.  With two barriers per
// iteration, every read of a ring precedes (through a barrier) the next iteration's writes to it, so
// the c_iy = +1 group needs 3 slots, c_iy = 0 two and c_iy = -1 one: 6 slots of 3 planes per ring.
constexpr int kRing3Planes = 18;

// Plane of direction i for the row with index q (q >= 0: rows counted from a fixed origin below the
// piece) in a ring of 3 / 2 / 1 slots per group.
__device__ __forceinline__ int ring3_plane(int i, int q) {
    switch (i) {
        case 2: return (q % 3) * 3 + 0;
        case 5: return (q % 3) * 3 + 1;
        case 6: return (q % 3) * 3 + 2;
        case 0: return 9 + (q & 1) * 3 + 0;
        case 1: return 9 + (q & 1) * 3 + 1;
        case 3: return 9 + (q & 1) * 3 + 2;
        case 4: return 15;
        case 7: return 16;
        default: return 17;
    }
}

// Tuning of the three-step strips (as for the two-step strips: staged phase-A rows and the
// shared-memory share per SM; 0 = the largest), and the form of its collisions: packed pairs (0) or
// two scalar collisions per pair (1; FP32 pipe instead of the packed pipe).
#ifndef UQLB_STRIP3_PREFETCH_F32
#define UQLB_STRIP3_PREFETCH_F32 UQLB_STRIP_PREFETCH_F32
#endif
#ifndef UQLB_STRIP3_PREFETCH_16
#define UQLB_STRIP3_PREFETCH_16 UQLB_STRIP_PREFETCH_16
#endif
#ifndef UQLB_STRIP3_CARVEOUT_F32_KB
#define UQLB_STRIP3_CARVEOUT_F32_KB UQLB_STRIP_CARVEOUT_F32_KB
#endif
#ifndef UQLB_STRIP3_CARVEOUT_16_KB
#define UQLB_STRIP3_CARVEOUT_16_KB UQLB_STRIP_CARVEOUT_16_KB
#endif
#ifndef UQLB_STRIP3_COLLIDE
#define UQLB_STRIP3_COLLIDE 0
#endif
__device__ __forceinline__ void strip3_collide(f2 (&g)[9], float omega, const PackedBGK& omega2, f2* usq) {
    if constexpr (UQLB_STRIP3_COLLIDE == 0) {
        collide_packed(g, omega2, usq);
    } else {
        float a[9], b[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) upk(g[i], a[i], b[i]);
        float qa = 0.0f, qb = 0.0f;
        collide_pair_scalar(a, b, omega, usq != nullptr ? &qa : nullptr, usq != nullptr ? &qb : nullptr);
        if (usq != nullptr) *usq = pk(qa, qb);
#pragma unroll
        for (int i = 0; i < 9; ++i) g[i] = pk(a[i], b[i]);
    }
}

template <typename S>
struct Strip3Tune {
    static constexpr int depth = sizeof(S) == 4 ? UQLB_STRIP3_PREFETCH_F32 : UQLB_STRIP3_PREFETCH_16;
    static constexpr int carveout_kb = sizeof(S) == 4 ? UQLB_STRIP3_CARVEOUT_F32_KB : UQLB_STRIP3_CARVEOUT_16_KB;
    static constexpr int max_nx_raw = (232448 - 2048) / (2 * kRing3Planes * 4 + depth * 9 * (int)sizeof(S)) / 64 * 64;
    static constexpr int max_nx = max_nx_raw < 2048 ? max_nx_raw : 2048;
};

template <typename S, bool GENERIC>
__global__ void __launch_bounds__(1024, 1) strip3_kernel(KParams p) {
    extern __shared__ __align__(16) unsigned char s4_raw[];
    __shared__ __align__(16) SampleDev s_sp;
    __shared__ int s_j, s_rows, s_nact, s_flag;
    const int tid = threadIdx.x, np = blockDim.x;
    const int rw = 2 * np;
    float* ring1 = reinterpret_cast<float*>(s4_raw);  // [kRing3Planes][rw]
    float* ring2 = ring1 + kRing3Planes * rw;         // [kRing3Planes][rw]
    double* s_red = reinterpret_cast<double*>(s4_raw);  // block sums: the rings, once a piece is done
    S* stage = reinterpret_cast<S*>(ring2 + kRing3Planes * rw);  // [D][9][rw]
    const int t = (int)p.step_counter[0] + p.dt;
    const int t0 = (int)p.step_counter[1];
    if (tid == 0) {
        const int nact = active_samples(p, t);
        s_nact = nact;
        s_rows = p.row_base[nact];
    }
    __syncthreads();
    const int nact = s_nact, rows = s_rows;
    const int per = (rows + gridDim.x - 1) / gridDim.x;
    const int r0 = blockIdx.x * per, r1 = min(rows, r0 + per);
    const bool series = p.qoi_every > 0 && p.series != nullptr;
    const bool sr = sizeof(S) == 2 && p.stochastic != 0;
    const int nx = GENERIC ? __ldg(&p.samples[0].nx) : rw;
    const int x = 2 * tid;
    const bool va = !GENERIC || x < nx, vb = !GENERIC || x + 1 < nx;
    const int xl = x == 0 ? nx - 1 : x - 1;
    const int xar = GENERIC && x + 1 >= nx ? x + 1 - nx : x + 1;
    const int xbr = x + 2 >= nx ? x + 2 - nx : x + 2;
    constexpr int D = Strip3Tune<S>::depth;
    for (int r = r0; r < r1;) {
        __syncthreads();  // the previous piece's ring reads and block sums are done
        if (tid == 0) {
            int lo = 0, hi = nact - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (p.row_base[mid] <= r)
                    lo = mid;
                else
                    hi = mid - 1;
            }
            s_j = lo;
        }
        __syncthreads();
        const int j = s_j;
        if (tid < 32) reinterpret_cast<uint32_t*>(&s_sp)[tid] = __ldg(reinterpret_cast<const uint32_t*>(p.samples + j) + tid);
        __syncthreads();
        const int rb = p.row_base[j];
        const int ny = s_sp.ny, pitch = s_sp.pitch, plane = (int)s_sp.plane;
        const int ya = r - rb, yb = min(ny, r1 - rb);
        r = rb + yb;
        const int n = min(3, s_sp.steps - t);  // steps of this launch for this sample (>= 1)
        bool want[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) want[k] = series && k < n && ((t + k) % p.qoi_every) == 0;
        const bool second = ((p.sel[s_sp.slot] ^ ((t - t0) / 3)) & 1) != 0;
        const S* src = static_cast<const S*>(second ? p.arena2 : p.arena) + s_sp.f_off;
        S* dst = static_cast<S*>(second ? p.arena : p.arena2) + s_sp.f_off;
        const float omega = (float)s_sp.omega;
        const PackedBGK omega2 = packed_bgk(omega);
        const uint32_t sid = (uint32_t)s_sp.sample_id;
        const typename Storage<S>::Q qz = quanta_of<S>(p, j);
        double red[3] = {0.0, 0.0, 0.0};
        // periodic row of a phase-A row (at most two rows outside the sample; samples have >= 2 rows,
        // two corrections each way keep any height in range)
        auto wrap = [&](int y) {
            y += y < 0 ? ny : 0;
            y += y < 0 ? ny : 0;
            y -= y >= ny ? ny : 0;
            y -= y >= ny ? ny : 0;
            return y;
        };
        // push of the pair's post-collision populations g (step ts, row y) into dst
        auto push = [&](int y, int ts, const f2 (&g)[9]) {
            const int ym = y == 0 ? ny - 1 : y - 1, yp = y == ny - 1 ? 0 : y + 1;
            const int row[3] = {ym * pitch, y * pitch, yp * pitch};
            if constexpr (sizeof(S) == 2) {
                // 16-bit storage: each population's pair rounded into one word (one hash per pair and
                // step for the stochastic bits), stored whole where it stays in its columns
                uint32_t h = 0u;
                if (sr)
                    h = mix32((uint32_t)(y * pitch + x) * 0x9E3779B1u + (uint32_t)ts * 0x85EBCA77u +
                              sid * 0xC2B2AE3Du);
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    S* d = dst + (i * plane + row[1 + cy(i)]);
                    const uint32_t w =
                        sr ? pair_word_sr<S>(g[i], sr_bits(h, i), qz, i) : pair_word<S>(g[i], qz, i);
                    if (cx(i) == 0 && vb) {
                        *reinterpret_cast<uint32_t*>(d + x) = w;
                    } else {
                        const int ca = cx(i) == 0 ? x : (cx(i) > 0 ? xar : xl);
                        const int cb = cx(i) == 0 ? x + 1 : (cx(i) > 0 ? xbr : x);
                        *reinterpret_cast<uint16_t*>(d + ca) = (uint16_t)w;
                        if (vb) *reinterpret_cast<uint16_t*>(d + cb) = (uint16_t)(w >> 16);
                    }
                }
            } else {
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    S* d = dst + (i * plane + row[1 + cy(i)]);
                    float a, b;
                    upk(g[i], a, b);
                    const int ca = cx(i) == 0 ? x : (cx(i) > 0 ? xar : xl);
                    const int cb = cx(i) == 0 ? x + 1 : (cx(i) > 0 ? xbr : x);
                    if (cx(i) == 0 && vb) {
                        pair_store<S>(d + x, g[i], qz, i);
                    } else {
                        Storage<S>::store(d + ca, a, qz, i);
                        if (vb) Storage<S>::store(d + cb, b, qz, i);
                    }
                }
            }
        };
        auto add_usq = [&](double& acc, f2 q) {
            float a, b;
            upk(q, a, b);
            acc += (double)a;
            if (vb) acc += (double)b;
        };
        // gather of row y's pair from a ring (population i from ring row y - c_iy, column x - c_ix);
        // oq: ring row index of row y (rows y - 1 and y + 1 are oq - 1 and oq + 1)
        auto gather = [&](const float* ring, int oq, f2 (&g)[9]) {
            const float* rp = ring + ring3_plane(2, oq - 1) * rw;  // c_iy = +1: row y - 1 (planes 2, 5, 6)
            const float* rz = ring + ring3_plane(0, oq) * rw;      // c_iy =  0: row y     (planes 0, 1, 3)
            const float* rm = ring + ring3_plane(4, oq + 1) * rw;  // c_iy = -1: row y + 1 (planes 4, 7, 8)
            g[0] = *reinterpret_cast<const f2*>(rz + x);
            g[1] = pk(rz[rw + xl], rz[rw + x]);
            g[3] = pk(rz[2 * rw + xar], rz[2 * rw + xbr]);
            g[2] = *reinterpret_cast<const f2*>(rp + x);
            g[5] = pk(rp[rw + xl], rp[rw + x]);
            g[6] = pk(rp[2 * rw + xar], rp[2 * rw + xbr]);
            g[4] = *reinterpret_cast<const f2*>(rm + x);
            g[7] = pk(rm[rw + xar], rm[rw + xbr]);
            g[8] = pk(rm[2 * rw + xl], rm[2 * rw + x]);
        };
        auto put_ring = [&](float* ring, int oq, const f2 (&g)[9]) {
            f2* r2 = reinterpret_cast<f2*>(ring);
#pragma unroll
            for (int i = 0; i < 9; ++i) r2[ring3_plane(i, oq) * np + tid] = g[i];
        };
        if (n == 1) {
            // the sample's last step: collide and push row by row
            for (int y = ya; y < yb && va; ++y) {
                const S* s0 = src + (y * pitch + x);
                f2 g[9];
#pragma unroll
                for (int i = 0; i < 9; ++i) g[i] = pair_load<S>(s0 + i * plane, qz, i);
                f2 q;
                strip3_collide(g, omega, omega2, want[0] ? &q : nullptr);
                if (want[0]) add_usq(red[0], q);
                push(y, t, g);
            }
        } else {
            // phase-A rows run from ya - (n == 3 ? 2 : 1) to yb + n - 2; ring row index of row y:
            // y - ya + 4 (>= 0 for every row the piece touches)
            const int a0 = ya - (n - 1);
            auto fetch = [&](int qa) {
                // staging: phase-A row a0 + qa goes to buffer qa % D, D rows ahead of its phase A; one
                // copy group per row (empty past the piece)
                if (va && a0 + qa <= yb + n - 2) {
                    const S* s0 = src + (wrap(a0 + qa) * pitch + x);
                    S* st = stage + (qa % (D > 0 ? D : 1)) * 9 * rw + x;
#pragma unroll
                    for (int i = 0; i < 9; ++i) cp_async<2 * sizeof(S)>(st + i * rw, s0 + i * plane);
                }
                cp_async_commit();
            };
            (void)fetch;
            auto phase_a = [&](int ya_row) {
                if (!va) return;
                const int qa = ya_row - a0;
                f2 g[9];
                if constexpr (D > 0) {
                    cp_async_wait<D - 1>();
                    const S* st = stage + (qa % D) * 9 * rw + x;
#pragma unroll
                    for (int i = 0; i < 9; ++i) g[i] = pair_load<S>(st + i * rw, qz, i);
                    fetch(qa + D);
                } else {
                    const S* s0 = src + (wrap(ya_row) * pitch + x);
#pragma unroll
                    for (int i = 0; i < 9; ++i) g[i] = pair_load<S>(s0 + i * plane, qz, i);
                }
                f2 qq;
                const bool w = want[0] && ya_row >= ya && ya_row < yb;
                strip3_collide(g, omega, omega2, w ? &qq : nullptr);
                if (w) add_usq(red[0], qq);
                put_ring(ring1, ya_row - ya + 4, g);
            };
#pragma unroll
            for (int k = 0; k < D; ++k) fetch(k);
            if (n == 3) {
                phase_a(ya - 2);
                phase_a(ya - 1);
                for (int y = ya - 2; y < yb; ++y) {
                    phase_a(y + 2);
                    __syncthreads();
                    if (va) {
                        // phase B: row y + 1 at step t + 1 from ring 1, into ring 2
                        f2 g[9];
                        gather(ring1, y + 1 - ya + 4, g);
                        f2 qq;
                        const bool w = want[1] && y + 1 >= ya && y + 1 < yb;
                        strip3_collide(g, omega, omega2, w ? &qq : nullptr);
                        if (w) add_usq(red[1], qq);
                        put_ring(ring2, y + 1 - ya + 4, g);
                    }
                    __syncthreads();
                    if (va && y >= ya) {
                        // phase C: row y at step t + 2 from ring 2, pushed into the other lattice
                        f2 g[9];
                        gather(ring2, y - ya + 4, g);
                        f2 qq;
                        strip3_collide(g, omega, omega2, want[2] ? &qq : nullptr);
                        if (want[2]) add_usq(red[2], qq);
                        push(y, t + 2, g);
                    }
                }
            } else {
                phase_a(ya - 1);
                for (int y = ya - 1; y < yb; ++y) {
                    phase_a(y + 1);
                    __syncthreads();
                    if (va && y >= ya) {
                        // phase B: row y at step t + 1 from ring 1, pushed into the other lattice
                        f2 g[9];
                        gather(ring1, y - ya + 4, g);
                        f2 qq;
                        strip3_collide(g, omega, omega2, want[1] ? &qq : nullptr);
                        if (want[1]) add_usq(red[1], qq);
                        push(y, t + 1, g);
                    }
                    __syncthreads();
                }
            }
            if constexpr (D > 0) cp_async_wait<0>();  // the empty groups past the piece
        }
        if (want[0] || want[1] || want[2]) {
            // this piece's sums; the block that completes the sample adds the pieces in row order
            __syncthreads();  // s_red lives in the rings
            block_sum_dyn<3>(red, s_red);
            if (tid == 0) {
#pragma unroll
                for (int k = 0; k < 3; ++k) p.partials[(int64_t)(rb + ya) * 3 + k] = red[k];
                __threadfence();
                const int prev = atomicAdd(p.counters + j, yb - ya);
                s_flag = (prev + (yb - ya) == ny);
            }
            __syncthreads();
            if (s_flag) {
                __threadfence();
                double acc[3] = {0.0, 0.0, 0.0};
                for (int q = tid; q < ny; q += np) {
                    if (q == 0 || (rb + q) % per == 0) {
#pragma unroll
                        for (int k = 0; k < 3; ++k) acc[k] += __ldcg(p.partials + (int64_t)(rb + q) * 3 + k);
                    }
                }
                block_sum_dyn<3>(acc, s_red);
                if (tid == 0) {
                    const int64_t row = (int64_t)s_sp.sample_id * p.series_ld;
#pragma unroll
                    for (int k = 0; k < 3; ++k)
                        if (want[k]) p.series[row + (t + k) / p.qoi_every] = acc[k] * s_sp.u_ref_inv2;
                    p.counters[j] = 0;
                }
            }
        }
    }
}


// ------------------------------------------------------------------------------------------
// Three-step strips at a compile-time width W (a whole number of 64-column blocks): the schedule of
// strip3_kernel with every shared-memory and global address an immediate offset from a few base
// pointers.  The rings keep two halo columns on each side of a row (RS = W + 4 floats per plane):
// the block's first and last pairs also write their values into the opposite halo, so the gathers of
// the edge columns read the periodic neighbours without any index wrapping.  The lattices keep each
// row's nine populations together (row stride 9 W, population stride W), so a row's loads and the
// push of its three destination rows are immediate offsets from one pointer per row.
// ------------------------------------------------------------------------------------------
// Threads per SM the register budget of the fixed-width strips is sized for (65536 registers over
// them).  Measured on the 625 x 256^2 ensemble (kernel GLUPS at 512 / 768 / 1024 threads): FP32 230 /
// 221 / 216 (four blocks fit the shared memory; more registers serve them best), FX16 167 / 190 / 195,
// BF16 185 / 201 / 212 (six blocks fit; the register budget then decides how many run).
#ifndef UQLB_STRIP3W_THREADS_F32
#define UQLB_STRIP3W_THREADS_F32 512
#endif
#ifndef UQLB_STRIP3W_THREADS_16
#define UQLB_STRIP3W_THREADS_16 1024
#endif
// Register staging (D == 2) holds nine more words per thread: 16-bit storage then takes the budget of
// 768 threads (85 registers; six blocks of 128 threads still fit), where 1024 would spill.
template <typename S, int D>
constexpr int strip3w_min_blocks(int np) {
    constexpr int th = sizeof(S) == 4 ? UQLB_STRIP3W_THREADS_F32 : (D == 2 ? 768 : UQLB_STRIP3W_THREADS_16);
    return th / np < 1 ? 1 : (th / np > 16 ? 16 : th / np);
}

// D: staging of the phase-A rows ahead of their use: 0 none, 1 the next row in shared memory
// (cp.async), 2 the next row in registers.
template <typename S, int W, int D>
__global__ void __launch_bounds__(W / 2, strip3w_min_blocks<S, D>(W / 2)) strip3w_kernel(KParams p) {
    constexpr int NP = W / 2, RS = W + 4;
    extern __shared__ __align__(16) unsigned char s5_raw[];
    __shared__ __align__(16) SampleDev s_sp;
    __shared__ int s_j, s_rows, s_nact, s_flag;
    const int tid = threadIdx.x;
    float* ring1 = reinterpret_cast<float*>(s5_raw);  // [kRing3Planes][RS]
    float* ring2 = ring1 + kRing3Planes * RS;
    double* s_red = reinterpret_cast<double*>(s5_raw);
    S* stage = reinterpret_cast<S*>(ring2 + kRing3Planes * RS);  // D == 1: [9][W], the next phase-A row
    const int t = (int)p.step_counter[0] + p.dt;
    const int t0 = (int)p.step_counter[1];
    if (tid == 0) {
        const int nact = active_samples(p, t);
        s_nact = nact;
        s_rows = p.row_base[nact];
    }
    __syncthreads();
    const int nact = s_nact, rows = s_rows;
    const int per = (rows + gridDim.x - 1) / gridDim.x;
    const int r0 = blockIdx.x * per, r1 = min(rows, r0 + per);
    const bool series = p.qoi_every > 0 && p.series != nullptr;
    const bool sr = sizeof(S) == 2 && p.stochastic != 0;
    const int x = 2 * tid;
    float* const r1t = ring1 + 2 + x;  // this thread's column x in ring 1 (column c sits at 2 + c)
    float* const r2t = ring2 + 2 + x;
    const bool first = tid == 0, last = tid == NP - 1;
    // push offsets of the wrapped neighbour columns: node a's x - 1 and node b's x + 2
    const int offl = first ? W - 1 : -1, offr = last ? 2 - W : 2;
    for (int r = r0; r < r1;) {
        __syncthreads();
        if (tid == 0) {
            int lo = 0, hi = nact - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (p.row_base[mid] <= r)
                    lo = mid;
                else
                    hi = mid - 1;
            }
            s_j = lo;
        }
        __syncthreads();
        const int j = s_j;
        if (tid < 32) reinterpret_cast<uint32_t*>(&s_sp)[tid] = __ldg(reinterpret_cast<const uint32_t*>(p.samples + j) + tid);
        __syncthreads();
        const int rb = p.row_base[j];
        const int ny = s_sp.ny;
        const int ya = r - rb, yb = min(ny, r1 - rb);
        r = rb + yb;
        const int n = min(3, s_sp.steps - t);
        bool want[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) want[k] = series && k < n && ((t + k) % p.qoi_every) == 0;
        const bool second = ((p.sel[s_sp.slot] ^ ((t - t0) / 3)) & 1) != 0;
        const S* src = static_cast<const S*>(second ? p.arena2 : p.arena) + s_sp.f_off + x;
        S* dst = static_cast<S*>(second ? p.arena : p.arena2) + s_sp.f_off + x;
        const float omega = (float)s_sp.omega;
        const PackedBGK omega2 = packed_bgk(omega);
        const uint32_t sid = (uint32_t)s_sp.sample_id;
        const typename Storage<S>::Q qz = quanta_of<S>(p, j);
        double red[3] = {0.0, 0.0, 0.0};
        auto wrap = [&](int y) {
            y += y < 0 ? ny : 0;
            y += y < 0 ? ny : 0;
            y -= y >= ny ? ny : 0;
            y -= y >= ny ? ny : 0;
            return y;
        };
        // FP32 stores (16-bit storage rounds whole pairs, in push)
        auto st1 = [&](S* d, float v, int i) { Storage<S>::store(d, v, qz, i); };
        auto st2 = [&](S* d, f2 v, int i) { pair_store<S>(d, v, qz, i); };
        // push of the pair's post-collision populations g (step ts, row y) into the other lattice
        auto push = [&](int y, int ts, const f2 (&g)[9]) {
            const int ym = y == 0 ? ny - 1 : y - 1, yp = y == ny - 1 ? 0 : y + 1;
            if constexpr (sizeof(S) == 2) {
                // 16-bit storage: each population's pair rounded into one word (one hash per pair and
                // step for the stochastic bits); the x-moving populations land in two columns
                uint32_t h = 0u;
                if (sr)
                    h = mix32((uint32_t)(y * 9 * W + x) * 0x9E3779B1u + (uint32_t)ts * 0x85EBCA77u +
                              sid * 0xC2B2AE3Du);
                auto word = [&](int i) {
                    return sr ? pair_word_sr<S>(g[i], sr_bits(h, i), qz, i) : pair_word<S>(g[i], qz, i);
                };
                auto put2 = [](S* at, uint32_t w) { *reinterpret_cast<uint32_t*>(at) = w; };
                auto put_lo = [](S* at, uint32_t w) { *reinterpret_cast<uint16_t*>(at) = (uint16_t)w; };
                auto put_hi = [](S* at, uint32_t w) { *reinterpret_cast<uint16_t*>(at) = (uint16_t)(w >> 16); };
                uint32_t w;
                {  // row y: populations 0, 1, 3
                    S* R = dst + y * (9 * W);
                    put2(R, word(0));
                    w = word(1);
                    put_lo(R + W + 1, w);
                    put_hi(R + offr + W, w);
                    w = word(3);
                    put_lo(R + offl + 3 * W, w);
                    put_hi(R + 3 * W, w);
                }
                {  // row y + 1: populations 2, 5, 6
                    S* R = dst + yp * (9 * W);
                    put2(R + 2 * W, word(2));
                    w = word(5);
                    put_lo(R + 5 * W + 1, w);
                    put_hi(R + offr + 5 * W, w);
                    w = word(6);
                    put_lo(R + offl + 6 * W, w);
                    put_hi(R + 6 * W, w);
                }
                {  // row y - 1: populations 4, 7, 8
                    S* R = dst + ym * (9 * W);
                    put2(R + 4 * W, word(4));
                    w = word(7);
                    put_lo(R + offl + 7 * W, w);
                    put_hi(R + 7 * W, w);
                    w = word(8);
                    put_lo(R + 8 * W + 1, w);
                    put_hi(R + offr + 8 * W, w);
                }
            } else {
                float a, b;
                {  // row y: populations 0, 1, 3
                    S* R = dst + y * (9 * W);
                    st2(R, g[0], 0);
                    upk(g[1], a, b);
                    st1(R + W + 1, a, 1);
                    st1(R + offr + W, b, 1);
                    upk(g[3], a, b);
                    st1(R + offl + 3 * W, a, 3);
                    st1(R + 3 * W, b, 3);
                }
                {  // row y + 1: populations 2, 5, 6
                    S* R = dst + yp * (9 * W);
                    st2(R + 2 * W, g[2], 2);
                    upk(g[5], a, b);
                    st1(R + 5 * W + 1, a, 5);
                    st1(R + offr + 5 * W, b, 5);
                    upk(g[6], a, b);
                    st1(R + offl + 6 * W, a, 6);
                    st1(R + 6 * W, b, 6);
                }
                {  // row y - 1: populations 4, 7, 8
                    S* R = dst + ym * (9 * W);
                    st2(R + 4 * W, g[4], 4);
                    upk(g[7], a, b);
                    st1(R + offl + 7 * W, a, 7);
                    st1(R + 7 * W, b, 7);
                    upk(g[8], a, b);
                    st1(R + 8 * W + 1, a, 8);
                    st1(R + offr + 8 * W, b, 8);
                }
            }
        };
        auto add_usq = [&](double& acc, f2 q) {
            float a, b;
            upk(q, a, b);
            acc += (double)a + (double)b;
        };
        // ring plane offsets of row index q: the c_y = +1 / 0 / -1 groups (3 / 2 / 1 slots)
        auto slot_p = [](int q) { return (q % 3) * 3 * RS; };
        auto slot_z = [](int q) { return (9 + (q & 1) * 3) * RS; };
        // the halo copy of the block's first pair (right halo: columns 0, 1 after W - 1) and last pair
        // (left halo: columns W - 2, W - 1 before 0)
        const int hoff = first ? W : -W;
        auto put_ring = [&](float* rt, int q, const f2 (&g)[9]) {
            const int op = slot_p(q), oz = slot_z(q), om = 15 * RS;
            auto put = [&](float* at, int off, f2 v) { *reinterpret_cast<f2*>(at + off) = v; };
            put(rt, op, g[2]);
            put(rt, op + RS, g[5]);
            put(rt, op + 2 * RS, g[6]);
            put(rt, oz, g[0]);
            put(rt, oz + RS, g[1]);
            put(rt, oz + 2 * RS, g[3]);
            put(rt, om, g[4]);
            put(rt, om + RS, g[7]);
            put(rt, om + 2 * RS, g[8]);
            if (first || last) {
                float* h = rt + hoff;
                put(h, op, g[2]);
                put(h, op + RS, g[5]);
                put(h, op + 2 * RS, g[6]);
                put(h, oz, g[0]);
                put(h, oz + RS, g[1]);
                put(h, oz + 2 * RS, g[3]);
                put(h, om, g[4]);
                put(h, om + RS, g[7]);
                put(h, om + 2 * RS, g[8]);
            }
        };
        // gather of row index q (population i from row q - c_iy, column x - c_ix)
        auto gather = [&](const float* rt, int q, f2 (&g)[9]) {
            const float* pp = rt + slot_p(q - 1);
            const float* pz = rt + slot_z(q);
            const float* pm = rt + 15 * RS;
            g[0] = *reinterpret_cast<const f2*>(pz);
            g[1] = pk(pz[RS - 1], pz[RS]);
            g[3] = pk(pz[2 * RS + 1], pz[2 * RS + 2]);
            g[2] = *reinterpret_cast<const f2*>(pp);
            g[5] = pk(pp[RS - 1], pp[RS]);
            g[6] = pk(pp[2 * RS + 1], pp[2 * RS + 2]);
            g[4] = *reinterpret_cast<const f2*>(pm);
            g[7] = pk(pm[RS + 1], pm[RS + 2]);
            g[8] = pk(pm[2 * RS - 1], pm[2 * RS]);
        };
        if (n == 1) {
            for (int y = ya; y < yb; ++y) {
                const S* s0 = src + y * (9 * W);
                f2 g[9];
#pragma unroll
                for (int i = 0; i < 9; ++i) g[i] = pair_load<S>(s0 + i * W, qz, i);
                f2 q;
                collide_packed(g, omega2, want[0] ? &q : nullptr);
                if (want[0]) add_usq(red[0], q);
                push(y, t, g);
            }
        } else {
            const int a0 = ya - (n - 1);
            auto fetch = [&](int qa) {
                if (a0 + qa <= yb + n - 2) {
                    const S* s0 = src + wrap(a0 + qa) * (9 * W);
                    S* st = stage + x;
#pragma unroll
                    for (int i = 0; i < 9; ++i) cp_async<2 * sizeof(S)>(st + i * W, s0 + i * W);
                }
                cp_async_commit();
            };
            (void)fetch;
            // D == 2: the next phase-A row's pairs are loaded into registers one row ahead, so their
            // latency overlaps the rest of the row's work and its barriers
            using Raw = PairRaw<S>;
            Raw pre[9];
            auto fetch_regs = [&](int row) {
                if (row - a0 <= yb + n - 2 - a0) {
                    const Raw* s0 = reinterpret_cast<const Raw*>(src + wrap(row) * (9 * W));
#pragma unroll
                    for (int i = 0; i < 9; ++i) pre[i] = __ldg(s0 + i * (W / 2));
                }
            };
            (void)fetch_regs;
            auto phase_a = [&](int row) {
                const int qa = row - a0;
                f2 g[9];
                if constexpr (D == 1) {
                    cp_async_wait<0>();
                    const S* st = stage + x;
#pragma unroll
                    for (int i = 0; i < 9; ++i) g[i] = pair_load<S>(st + i * W, qz, i);
                    fetch(qa + 1);
                } else if constexpr (D == 2) {
#pragma unroll
                    for (int i = 0; i < 9; ++i) g[i] = pair_from_raw<S>(pre[i], qz, i);
                    fetch_regs(row + 1);
                } else {
                    const S* s0 = src + wrap(row) * (9 * W);
#pragma unroll
                    for (int i = 0; i < 9; ++i) g[i] = pair_load<S>(s0 + i * W, qz, i);
                }
                f2 qq;
                const bool w = want[0] && row >= ya && row < yb;
                collide_packed(g, omega2, w ? &qq : nullptr);
                if (w) add_usq(red[0], qq);
                put_ring(r1t, row - ya + 4, g);
            };
            if constexpr (D == 1) fetch(0);
            if constexpr (D == 2) fetch_regs(a0);
            if (n == 3) {
                phase_a(ya - 2);
                phase_a(ya - 1);
                for (int y = ya - 2; y < yb; ++y) {
                    phase_a(y + 2);
                    __syncthreads();
                    {
                        f2 g[9];
                        gather(r1t, y + 1 - ya + 4, g);
                        f2 qq;
                        const bool w = want[1] && y + 1 >= ya && y + 1 < yb;
                        collide_packed(g, omega2, w ? &qq : nullptr);
                        if (w) add_usq(red[1], qq);
                        put_ring(r2t, y + 1 - ya + 4, g);
                    }
                    __syncthreads();
                    if (y >= ya) {
                        f2 g[9];
                        gather(r2t, y - ya + 4, g);
                        f2 qq;
                        collide_packed(g, omega2, want[2] ? &qq : nullptr);
                        if (want[2]) add_usq(red[2], qq);
                        push(y, t + 2, g);
                    }
                }
            } else {
                phase_a(ya - 1);
                for (int y = ya - 1; y < yb; ++y) {
                    phase_a(y + 1);
                    __syncthreads();
                    if (y >= ya) {
                        f2 g[9];
                        gather(r1t, y - ya + 4, g);
                        f2 qq;
                        collide_packed(g, omega2, want[1] ? &qq : nullptr);
                        if (want[1]) add_usq(red[1], qq);
                        push(y, t + 1, g);
                    }
                    __syncthreads();
                }
            }
            if constexpr (D == 1) cp_async_wait<0>();
        }
        if (want[0] || want[1] || want[2]) {
            __syncthreads();
            block_sum_dyn<3>(red, s_red);
            if (tid == 0) {
#pragma unroll
                for (int k = 0; k < 3; ++k) p.partials[(int64_t)(rb + ya) * 3 + k] = red[k];
                __threadfence();
                const int prev = atomicAdd(p.counters + j, yb - ya);
                s_flag = (prev + (yb - ya) == ny);
            }
            __syncthreads();
            if (s_flag) {
                __threadfence();
                double acc[3] = {0.0, 0.0, 0.0};
                for (int q = tid; q < ny; q += NP) {
                    if (q == 0 || (rb + q) % per == 0) {
#pragma unroll
                        for (int k = 0; k < 3; ++k) acc[k] += __ldcg(p.partials + (int64_t)(rb + q) * 3 + k);
                    }
                }
                block_sum_dyn<3>(acc, s_red);
                if (tid == 0) {
                    const int64_t row = (int64_t)s_sp.sample_id * p.series_ld;
#pragma unroll
                    for (int k = 0; k < 3; ++k)
                        if (want[k]) p.series[row + (t + k) / p.qoi_every] = acc[k] * s_sp.u_ref_inv2;
                    p.counters[j] = 0;
                }
            }
        }
    }
}


// ------------------------------------------------------------------------------------------
// Channel samples held on chip: one thread-block cluster per sample runs its whole time loop.
// ------------------------------------------------------------------------------------------
// The C blocks of a cluster split the sample's columns into C slabs of cw columns; each block keeps
// its slab's populations once in shared memory (row after row, each row the nine populations of the
// slab's columns padded to a compiled row width where it fits, in the storage type), so HBM is touched
// only to load the state at the start and to write it back at the end.  The steps alternate the
// two halves of the in-place AA order, counted from the run's first step: an even step reads a
// node's own nine slots, collides (BGK, the one-step kernel's formulas) and writes each
// post-collision population g*_i back into the node's own slot opp(i), already replaced by its
// boundary rule where link i meets a wall, the obstacle, the inlet or the outlet (halfway
// bounce-back, moving-wall inlet, pressure outlet with the node's own velocity); an odd step reads
// g*_i of every neighbour x - c_i from its slot opp(i) (its own slot i across a boundary link),
// collides, and writes g*_i into slot i of the neighbour x + c_i (its own slot opp(i), after the
// boundary rule, across a boundary link), so the state is back in natural layout.  A node reads and
// writes the same slots within a step, so no step needs a second copy.  Slots of a neighbouring slab
// are read and written in that block's shared memory (distributed shared memory of the cluster), at
// odd steps only.  The cluster synchronises once per step with the hardware cluster barrier, which
// every thread of every block reaches at every step (the step loop and the stop decision are uniform
// over the cluster), so no wait depends on a flag.  Link classes of every node are precomputed once
// into shared memory (3 bits per direction), and the fluid nodes listed by the path they take.
// The values equal the one-step kernel's: the same collisions, the same boundary rules, applied at
// the step of the collision.  Forces at the QoI steps: block sums in shared memory, added by block 0
// in rank order; block 0 records C_D and C_L and takes the steady-state decision, which every block
// reads after a second barrier.  Samples with the Bouzidi obstacle or the interpolated inlet/outlet
// take the one-step kernel instead.
__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ unsigned cluster_rank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ unsigned cluster_size() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ unsigned cluster_id_x() {
    unsigned r;
    asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
    return r;
}
#ifndef UQLB_CLUSTER_THREADS
#define UQLB_CLUSTER_THREADS 1024
#endif
constexpr int kClusterThreads = UQLB_CLUSTER_THREADS;
// Fixed part of a cluster step's time, in node updates of one block (see launch_cluster_any).
constexpr double kClusterStepFixed = 3400.0;

// Exclusive block-wide prefix sums of v[0..N) over the threads in index order (every thread of the
// block calls it); the totals into tot.  sm: N values per warp.
template <int N>
__device__ __forceinline__ void block_scan(int (&v)[N], int (&tot)[N], int (*sm)[N]) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int in[N];
#pragma unroll
    for (int c = 0; c < N; ++c) in[c] = v[c];
#pragma unroll
    for (int d = 1; d < 32; d <<= 1)
#pragma unroll
        for (int c = 0; c < N; ++c) {
            const int u = __shfl_up_sync(0xFFFFFFFFu, in[c], d);
            if (lane >= d) in[c] += u;
        }
    if (lane == 31)
#pragma unroll
        for (int c = 0; c < N; ++c) sm[w][c] = in[c];
    __syncthreads();
    if (w == 0) {
        int x[N];
#pragma unroll
        for (int c = 0; c < N; ++c) x[c] = lane < nw ? sm[lane][c] : 0;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1)
#pragma unroll
            for (int c = 0; c < N; ++c) {
                const int u = __shfl_up_sync(0xFFFFFFFFu, x[c], d);
                if (lane >= d) x[c] += u;
            }
        if (lane < nw)
#pragma unroll
            for (int c = 0; c < N; ++c) sm[lane][c] = x[c];
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < N; ++c) {
        tot[c] = sm[nw - 1][c];
        v[c] = (w > 0 ? sm[w - 1][c] : 0) + in[c] - v[c];
    }
    __syncthreads();
}

// 32-bit shared::cluster address of a shared-memory location of this block, in block `rank`.
__device__ __forceinline__ uint32_t cluster_addr(const void* p, unsigned rank) {
    uint32_t a = (uint32_t)__cvta_generic_to_shared(p), r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
    return r;
}
template <typename S>
__device__ __forceinline__ void st_cluster(uint32_t addr, S v) {
    if constexpr (sizeof(S) == 4) {
        asm volatile("st.shared::cluster.b32 [%0], %1;" ::"r"(addr), "r"(*reinterpret_cast<uint32_t*>(&v)) : "memory");
    } else {
        asm volatile("st.shared::cluster.b16 [%0], %1;" ::"r"(addr), "h"(*reinterpret_cast<unsigned short*>(&v)) : "memory");
    }
}
template <typename S>
__device__ __forceinline__ S ld_cluster(uint32_t addr) {
    S v;
    if constexpr (sizeof(S) == 4) {
        uint32_t r;
        asm volatile("ld.shared::cluster.b32 %0, [%1];" : "=r"(r) : "r"(addr) : "memory");
        v = *reinterpret_cast<S*>(&r);
    } else {
        unsigned short r;
        asm volatile("ld.shared::cluster.b16 %0, [%1];" : "=h"(r) : "r"(addr) : "memory");
        v = *reinterpret_cast<S*>(&r);
    }
    return v;
}
__device__ __forceinline__ double ld_cluster_f64(uint32_t addr) {
    double v;
    asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(addr) : "memory");
    return v;
}
__device__ __forceinline__ int ld_cluster_s32(uint32_t addr) {
    int v;
    asm volatile("ld.shared::cluster.s32 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
    return v;
}

// Columns a cluster block's rows hold for a slab of cw columns: the smallest compiled row width
// (16, 32, 48, 64) at least cw, 0 beyond 64.
__host__ __device__ constexpr int cluster_padded_width(int cw) {
    return cw <= 16 ? 16 : (cw <= 32 ? 32 : (cw <= 48 ? 48 : (cw <= 64 ? 64 : 0)));
}

// Bytes of one slab state of ny rows of rw elements in a cluster block, rounded up to 16 (the link
// words follow it).
__host__ __device__ constexpr size_t cluster_state_bytes(int rw, int ny, int eb) {
    return ((size_t)rw * ny * eb + 15) / 16 * 16;
}
// Elements of storage type S that span the 32 four-byte shared-memory banks.
template <typename S>
constexpr int cluster_bank_span = 128 / (int)sizeof(S);

// The cluster kernel's node pass: one copy per step parity (compile-time parity) or one copy with the
// parity tested per population.  UQLB_CLUSTER_SPLIT_PARITY 1: split, 0: not, 2: split for 16-bit
// storage only.  Measured (GLUPS, split / not): FP32 cylinder 56.1 / 57.9, BF16 channel samples of the
// uneven batch 57.4 / 53.6.
#ifndef UQLB_CLUSTER_SPLIT_PARITY
#define UQLB_CLUSTER_SPLIT_PARITY 2
#endif
template <typename S>
constexpr bool kClusterSplitParity = UQLB_CLUSTER_SPLIT_PARITY == 1 || (UQLB_CLUSTER_SPLIT_PARITY == 2 && sizeof(S) == 2);
template <typename S, int CW>
__global__ void __launch_bounds__(kClusterThreads, 1) cluster_kernel(KParams p) {
    extern __shared__ __align__(16) unsigned char s6_raw[];
    __shared__ __align__(16) SampleDev s_sp;
    __shared__ double s_red[(kClusterThreads / 32) * 2];
    __shared__ double s_force[2];   // this block's force partial of the step (read by block 0)
    __shared__ int s_stop;          // block 0: 1 once the sample stops
    __shared__ int s_scan[kClusterThreads / 32][4];
    using C = typename Storage<S>::C;
    const int tid = threadIdx.x;
    const unsigned rank = cluster_rank(), nrank = cluster_size();
    const int j = (int)cluster_id_x();  // sample (table order)
    if (tid < 32) reinterpret_cast<uint32_t*>(&s_sp)[tid] = __ldg(reinterpret_cast<const uint32_t*>(p.samples + j) + tid);
    if (tid == 0) s_stop = 0;
    __syncthreads();
    const SampleDev& sp = s_sp;
    // the sample's columns over the cluster's blocks (a sample narrower than the widest of the
    // launch takes narrower slabs; the shared memory is sized for the widest)
    const int nx = sp.nx, ny = sp.ny, cw = (nx + (int)nrank - 1) / (int)nrank;
    const int x0 = (int)rank * cw, ncol = max(0, min(cw, nx - x0));  // this block's columns [x0, x0 + ncol)
    // row width of the block's state: CW columns (compiled), or the slab's cw when CW is 0; the rows
    // lie RW elements apart, with RW = 9 RC padded on the compiled widths so that consecutive rows
    // start cw elements (mod the 32 banks' span) apart: a warp's list entries, which run over the end
    // of one row into the next, then take distinct banks as they would in one plane of cw columns
    const int RC = CW > 0 ? CW : cw;
    constexpr int M = cluster_bank_span<S>;
    const int RW = 9 * RC + (CW > 0 ? ((cw - 9 * RC) % M + M) % M : 0);
    // the state: population i of row y and column lx at y RW + i RC + lx (each row's nine populations
    // together, CW >= cw columns each, or cw), so the offset between any two slots a node touches is
    // a compile-time constant where CW is compiled
    S* const lat = reinterpret_cast<S*>(s6_raw);
    uint32_t* const links =
        reinterpret_cast<uint32_t*>(s6_raw + cluster_state_bytes(RW, ny, (int)sizeof(S)));  // [ny][RC]
    uint32_t* const list = links + ny * RC;  // the fluid nodes, (y << 16) | column, grouped by path
    const typename Storage<S>::Q qz = quanta_of<S>(p, j);
    const uint32_t* mask = sp.mask_off >= 0 ? p.masks + sp.mask_off : nullptr;
    S* glob = static_cast<S*>(p.arena) + sp.f_off;
    const int t0 = (int)p.step_counter[1];
    const int T = sp.steps;
    const bool skip = p.done[sp.slot] != 0 || t0 >= T;
    // load the state at t0 (natural layout) and classify the links of every owned node:
    // class of direction i in bits 3i..3i+2 (kInterior .. kSolid); solid nodes get all ones
    for (int n = tid; n < ny * ncol; n += kClusterThreads) {
        const int y = n / ncol, lx = n - y * ncol, x = x0 + lx;
        const int64_t own = (int64_t)y * sp.pitch + x;
#pragma unroll
        for (int i = 0; i < 9; ++i) lat[y * RW + i * RC + lx] = glob[i * sp.plane + own];
        uint32_t w = 0u;
        if (mask != nullptr && mask_solid(mask, mask_words(sp), x, y)) {
            w = 0xFFFFFFFFu;
        } else {
#pragma unroll
            for (int i = 1; i < 9; ++i) w |= (uint32_t)classify(sp, mask, x + cx(i), y + cy(i)) << (3 * i);
            // bit 0 (no direction uses bits 0..2): a node whose neighbours lie partly in another slab
            if (lx == 0 || lx == ncol - 1) w |= 1u;
        }
        links[y * RC + lx] = w;
    }
    // shared::cluster addresses of the neighbouring blocks' states (same layout everywhere)
    const unsigned left = rank > 0 ? rank - 1 : rank, right = rank + 1 < nrank ? rank + 1 : rank;
    const uint32_t nl = cluster_addr(lat, left), nr = cluster_addr(lat, right);
    cluster_sync_all();
    const C omega = (C)sp.omega;
    const bool sr = sizeof(S) == 2 && p.stochastic != 0;
    const uint32_t sid = (uint32_t)sp.sample_id;
    // The fluid nodes in four lists, each in row-major order: boundary nodes (a link that is not
    // interior: boundary rules), interior nodes at the slab's left and at its right edge (three
    // neighbours in the next slab) and the rest (every neighbour in this slab), so that a warp
    // seldom mixes two paths.  Each thread takes a contiguous run of nodes and a block-wide scan
    // places its entries: the lists, and with them every thread's force partial, are the same at
    // every run.
    const int nnodes = ny * ncol;
    int nk[4];  // list lengths
    {
        // list of a node from its link word (a one-column slab has both edges: boundary path)
        auto kind = [&](uint32_t w, int lx) {
            return w == 0xFFFFFFFFu ? -1 : (w == 0u ? 3 : (w == 1u && ncol > 1 ? (lx == 0 ? 1 : 2) : 0));
        };
        const int chunk = (nnodes + kClusterThreads - 1) / kClusterThreads;
        const int c0 = min(nnodes, tid * chunk), c1 = min(nnodes, c0 + chunk);
        int off[4] = {0, 0, 0, 0};
        for (int n = c0; n < c1; ++n) {
            const int y = n / ncol, lx = n - y * ncol, k = kind(links[y * RC + lx], lx);
#pragma unroll
            for (int c = 0; c < 4; ++c) off[c] += k == c;
        }
        block_scan<4>(off, nk, s_scan);
        int base[4];
        base[0] = 0;
#pragma unroll
        for (int c = 1; c < 4; ++c) base[c] = base[c - 1] + nk[c - 1];
#pragma unroll
        for (int c = 0; c < 4; ++c) off[c] += base[c];
        for (int n = c0; n < c1; ++n) {
            const int y = n / ncol, lx = n - y * ncol, k = kind(links[y * RC + lx], lx);
            const uint32_t e = ((uint32_t)y << 16) | (uint32_t)lx;
#pragma unroll
            for (int c = 0; c < 4; ++c)
                if (k == c) list[off[c]++] = e;
        }
        __syncthreads();
    }
    // list boundaries: [0, e0) boundary, [e0, e1) left edge, [e1, e2) right edge, [e2, e3) inner
    const int e0 = nk[0], e1 = e0 + nk[1], e2 = e1 + nk[2], e3 = e2 + nk[3];
    // shared::cluster address of slot i of row y in the left (column cw - 1) or right (column 0)
    // neighbouring slab
    auto remote = [&](bool to_left, int i, int y) {
        return to_left ? nl + (uint32_t)(y * RW + i * RC + cw - 1) * (uint32_t)sizeof(S)
                       : nr + (uint32_t)(y * RW + i * RC) * (uint32_t)sizeof(S);
    };
    // the incoming populations (stored values) of list entry k at an odd step: g*_i of the neighbour
    // x - c_i from its slot opp(i), or the node's own slot i across a boundary link (written there by
    // the even step)
    auto gather_odd = [&](int k, int yn, int xn, int own, uint32_t lw, S (&v)[9]) {
        v[0] = lat[own];
        if (k >= e2) {
#pragma unroll
            for (int i = 1; i < 9; ++i) v[i] = lat[own + opp(i) * RC - cy(i) * RW - cx(i)];
        } else if (k >= e0) {
            const bool at_left = k < e1;
#pragma unroll
            for (int i = 1; i < 9; ++i) {
                if (at_left ? cx(i) > 0 : cx(i) < 0)
                    v[i] = ld_cluster<S>(remote(at_left, opp(i), yn - cy(i)));
                else
                    v[i] = lat[own + opp(i) * RC - cy(i) * RW - cx(i)];
            }
        } else {
#pragma unroll
            for (int i = 1; i < 9; ++i) {
                const int sl = xn - cx(i), sy = yn - cy(i);
                if (((lw >> (3 * opp(i))) & 7u) != kInterior)
                    v[i] = lat[own + i * RC];
                else if (sl < 0 || sl >= ncol)
                    v[i] = ld_cluster<S>(remote(sl < 0, opp(i), sy));
                else
                    v[i] = lat[sy * RW + opp(i) * RC + sl];
            }
        }
    };
    int t = t0;
    for (; t < T && !skip; ++t) {
        const bool odd = ((t - t0) & 1) != 0;
        const bool f_step = p.qoi_every > 0 && ((t + 1) % p.qoi_every) == 0;
        double fx = 0.0, fy = 0.0;
        // work units of 32 list entries, one per lane: warp w takes unit w in the first round and unit
        // 32 r + 31 - w in round r >= 1.  The lists start with the costlier boundary and edge nodes,
        // so the warps that took those in the first round take no unit of a last, partial round.
        if constexpr (kClusterSplitParity<S>) {
            // the parity of the step is a compile-time branch of the node pass (one copy of the pass per
            // parity), so no per-population test of it remains
            auto node_pass = [&](auto parity) {
                constexpr bool ODD = decltype(parity)::value;
                const int lane = tid & 31, wid = tid >> 5;
                constexpr int NW = kClusterThreads / 32;
                for (int r = 0; r * NW * 32 < e3; ++r) {
                    const int k = (r * NW + (r == 0 ? wid : NW - 1 - wid)) * 32 + lane;
                    if (k >= e3) continue;
                    const uint32_t e = list[k];
                    const int yn = (int)(e >> 16), xn = (int)(e & 0xFFFFu), own = yn * RW + xn;
                    const uint32_t lw = k < e0 ? links[yn * RC + xn] : 0u;
                    C g[9];
                    if constexpr (ODD) {
                        S v[9];
                        gather_odd(k, yn, xn, own, lw, v);
#pragma unroll
                        for (int i = 0; i < 9; ++i) g[i] = Storage<S>::load(v + i, qz, i);
        
        } else {
#pragma unroll
                        for (int i = 0; i < 9; ++i) g[i] = Storage<S>::load(lat + own + i * RC, qz, i);
                    }
                    C drho, jx, jy, ux, uy;
                    moments(g, drho, jx, jy, ux, uy);
                    bgk(g, omega, drho, jx, jy, ux, uy);
                    const uint32_t h = sr ? mix32((uint32_t)((int64_t)yn * sp.pitch + x0 + xn) * 0x9E3779B1u +
                                                  (uint32_t)t * 0x85EBCA77u + sid * 0xC2B2AE3Du)
                                          : 0u;
                    // the stored value of population i (rounded as the storage rounds)
                    auto cvt = [&](C v, int i) {
                        S r;
                        if (sr)
                            Storage<S>::store_sr(&r, v, (h * (0x2545F491u + 0x6A09E668u * (uint32_t)i)) >> 16, qz, i);
                        else
                            Storage<S>::store(&r, v, qz, i);
                        return r;
                    };
                    if (k >= e0) {
                        // every link interior: even steps write g*_i into the node's slot opp(i), odd steps
                        // into slot i of the neighbour x + c_i (across the slab's edge for the three
                        // populations of an edge node that leave it)
                        lat[own] = cvt(g[0], 0);
                        const bool edge = k < e2, at_left = k < e1;
#pragma unroll
                        for (int i = 1; i < 9; ++i) {
                            if constexpr (!ODD)
                                lat[own + opp(i) * RC] = cvt(g[i], i);
                            else if (edge && (at_left ? cx(i) < 0 : cx(i) > 0))
                                st_cluster<S>(remote(at_left, i, yn + cy(i)), cvt(g[i], i));
                            else
                                lat[own + i * RC + cy(i) * RW + cx(i)] = cvt(g[i], i);
                        }
                        continue;
                    }
                    lat[own] = cvt(g[0], 0);
#pragma unroll
                    for (int i = 1; i < 9; ++i) {
                        const int cls = (lw >> (3 * i)) & 7;
                        const int o = opp(i);
                        if (cls == kInterior) {
                            if constexpr (!ODD) {
                                lat[own + o * RC] = cvt(g[i], i);
                            } else {
                                const int dl = xn + cx(i), dy = yn + cy(i);
                                if (dl >= 0 && dl < ncol)
                                    lat[dy * RW + i * RC + dl] = cvt(g[i], i);
                                else
                                    st_cluster<S>(remote(dl < 0, i, dy), cvt(g[i], i));
                            }
                        } else if (cls == kWall || cls == kSolid) {
                            lat[own + o * RC] = cvt(g[i], i);
                            if (f_step && cls == kSolid) {
                                const C fs = g[i] + wgt<C>(i);
                                fx += (double)(C(2 * cx(i)) * fs);
                                fy += (double)(C(2 * cy(i)) * fs);
                            }
                        } else if (cls == kInlet) {
                            const C yy = C(yn) + C(0.5) - C(0.5) * C(cy(o));
                            lat[own + o * RC] = cvt(g[i] + C(6) * wgt<C>(o) * C(cx(o)) * inflow<C>(sp, yy, t), i);
                        } else {
                            const C cu = C(cx(o)) * ux + C(cy(o)) * uy;
                            lat[own + o * RC] = cvt(-g[i] + wgt<C>(o) * (C(9) * cu * cu - C(3) * (ux * ux + uy * uy)), i);
                        }
                    }
                }
            };
            if (odd)
                node_pass(std::true_type{});
            else
                node_pass(std::false_type{});
            } else {
            const int lane = tid & 31, wid = tid >> 5;
            constexpr int NW = kClusterThreads / 32;
            for (int r = 0; r * NW * 32 < e3; ++r) {
                const int k = (r * NW + (r == 0 ? wid : NW - 1 - wid)) * 32 + lane;
                if (k >= e3) continue;
                const uint32_t e = list[k];
                const int yn = (int)(e >> 16), xn = (int)(e & 0xFFFFu), own = yn * RW + xn;
                const uint32_t lw = k < e0 ? links[yn * RC + xn] : 0u;
                C g[9];
                if (odd) {
                    S v[9];
                    gather_odd(k, yn, xn, own, lw, v);
#pragma unroll
                    for (int i = 0; i < 9; ++i) g[i] = Storage<S>::load(v + i, qz, i);
                } else {
#pragma unroll
                    for (int i = 0; i < 9; ++i) g[i] = Storage<S>::load(lat + own + i * RC, qz, i);
                }
                C drho, jx, jy, ux, uy;
                moments(g, drho, jx, jy, ux, uy);
                bgk(g, omega, drho, jx, jy, ux, uy);
                const uint32_t h = sr ? mix32((uint32_t)((int64_t)yn * sp.pitch + x0 + xn) * 0x9E3779B1u +
                                              (uint32_t)t * 0x85EBCA77u + sid * 0xC2B2AE3Du)
                                      : 0u;
                // the stored value of population i (rounded as the storage rounds)
                auto cvt = [&](C v, int i) {
                    S r;
                    if (sr)
                        Storage<S>::store_sr(&r, v, (h * (0x2545F491u + 0x6A09E668u * (uint32_t)i)) >> 16, qz, i);
                    else
                        Storage<S>::store(&r, v, qz, i);
                    return r;
                };
                if (k >= e0) {
                    // every link interior: even steps write g*_i into the node's slot opp(i), odd steps
                    // into slot i of the neighbour x + c_i (across the slab's edge for the three
                    // populations of an edge node that leave it)
                    lat[own] = cvt(g[0], 0);
                    const bool edge = k < e2, at_left = k < e1;
#pragma unroll
                    for (int i = 1; i < 9; ++i) {
                        if (!odd)
                            lat[own + opp(i) * RC] = cvt(g[i], i);
                        else if (edge && (at_left ? cx(i) < 0 : cx(i) > 0))
                            st_cluster<S>(remote(at_left, i, yn + cy(i)), cvt(g[i], i));
                        else
                            lat[own + i * RC + cy(i) * RW + cx(i)] = cvt(g[i], i);
                    }
                    continue;
                }
                lat[own] = cvt(g[0], 0);
#pragma unroll
                for (int i = 1; i < 9; ++i) {
                    const int cls = (lw >> (3 * i)) & 7;
                    const int o = opp(i);
                    if (cls == kInterior) {
                        if (!odd) {
                            lat[own + o * RC] = cvt(g[i], i);
                        } else {
                            const int dl = xn + cx(i), dy = yn + cy(i);
                            if (dl >= 0 && dl < ncol)
                                lat[dy * RW + i * RC + dl] = cvt(g[i], i);
                            else
                                st_cluster<S>(remote(dl < 0, i, dy), cvt(g[i], i));
                        }
                    } else if (cls == kWall || cls == kSolid) {
                        lat[own + o * RC] = cvt(g[i], i);
                        if (f_step && cls == kSolid) {
                            const C fs = g[i] + wgt<C>(i);
                            fx += (double)(C(2 * cx(i)) * fs);
                            fy += (double)(C(2 * cy(i)) * fs);
                        }
                    } else if (cls == kInlet) {
                        const C yy = C(yn) + C(0.5) - C(0.5) * C(cy(o));
                        lat[own + o * RC] = cvt(g[i] + C(6) * wgt<C>(o) * C(cx(o)) * inflow<C>(sp, yy, t), i);
                    } else {
                        const C cu = C(cx(o)) * ux + C(cy(o)) * uy;
                        lat[own + o * RC] = cvt(-g[i] + wgt<C>(o) * (C(9) * cu * cu - C(3) * (ux * ux + uy * uy)), i);
                    }
                }
            }
        }
        if (f_step) {
            double v[2] = {fx, fy};
            block_sum<2, kClusterThreads>(v, s_red);
            if (tid == 0) {
                s_force[0] = v[0];
                s_force[1] = v[1];
            }
        }
        cluster_sync_all();  // the step is complete in every block
        if (f_step) {
            if (rank == 0 && tid == 0) {
                double F[2] = {0.0, 0.0};
                for (unsigned r = 0; r < nrank; ++r) {
                    const uint32_t a = cluster_addr(s_force, r);
                    F[0] += ld_cluster_f64(a);
                    F[1] += ld_cluster_f64(a + 8u);
                }
                record_force(p, sp, j, t + 1, F[0], F[1]);
                s_stop = p.done[sp.slot];
            }
            cluster_sync_all();  // block 0's decision is visible
            if (ld_cluster_s32(cluster_addr(&s_stop, 0u)) != 0) {
                ++t;
                break;
            }
        }
    }
    // the state at the last step run back to the arena in natural layout: after an odd number of
    // steps the slots hold the post-collision values of an even step, so each fluid node gathers its
    // incoming populations as an odd step would
    if (!skip) {
        if (((t - t0) & 1) != 0) {
            for (int k = tid; k < e3; k += kClusterThreads) {
                const uint32_t e = list[k];
                const int yn = (int)(e >> 16), xn = (int)(e & 0xFFFFu), own = yn * RW + xn;
                S v[9];
                gather_odd(k, yn, xn, own, k < e0 ? links[yn * RC + xn] : 0u, v);
                const int64_t at = (int64_t)yn * sp.pitch + x0 + xn;
#pragma unroll
                for (int i = 0; i < 9; ++i) glob[i * sp.plane + at] = v[i];
            }
            for (int n = tid; n < ny * ncol; n += kClusterThreads) {
                const int y = n / ncol, lx = n - y * ncol;
                if (links[y * RC + lx] != 0xFFFFFFFFu) continue;
                const int64_t at = (int64_t)y * sp.pitch + x0 + lx;
#pragma unroll
                for (int i = 0; i < 9; ++i) glob[i * sp.plane + at] = lat[y * RW + i * RC + lx];
            }
        } else {
            for (int n = tid; n < ny * ncol; n += kClusterThreads) {
                const int y = n / ncol, lx = n - y * ncol;
                const int64_t at = (int64_t)y * sp.pitch + x0 + lx;
#pragma unroll
                for (int i = 0; i < 9; ++i) glob[i * sp.plane + at] = lat[y * RW + i * RC + lx];
            }
        }
        if (rank == 0 && tid == 0 && !p.done[sp.slot]) p.steps_run[sp.slot] = t;
    }
    cluster_sync_all();  // no block leaves while another may still read its shared memory
}

// Shared memory of a cluster block whose rows hold CW columns (0: the slab's cw) for slabs of up to cw
// columns and ny rows (state, link words, node list).
template <typename S>
size_t cluster_smem(int CW, int cw, int ny) {
    // compiled width: rows of 9 CW elements plus the largest bank padding; else rows of 9 cw
    const int rw = CW > 0 ? 9 * CW + cluster_bank_span<S> - 1 : 9 * cw, rc = CW > 0 ? CW : cw;
    return cluster_state_bytes(rw, ny, (int)sizeof(S)) + (size_t)2 * rc * ny * sizeof(uint32_t);
}
constexpr size_t kClusterSmemMax = 227 * 1024 - 4096;
// Row width of the launch for slabs of cw columns and ny rows: the padded compiled width where its
// shared memory fits, else 0 (rows of exactly cw columns, strides at run time).
template <typename S>
int cluster_row_width(int cw, int ny) {
    const int w = cluster_padded_width(cw);
    return w > 0 && cluster_smem<S>(w, cw, ny) <= kClusterSmemMax ? w : 0;
}

template <typename S, int CW>
cudaError_t launch_cluster_w(const KParams& p, const BatchGeometry& g, cudaStream_t s, bool prepare_only) {
    const int csize = p.cluster_size;
    const size_t smem = cluster_smem<S>(CW, p.cluster_cw, p.cluster_ny);
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(cluster_kernel<S, CW>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        cudaFuncSetAttribute(cluster_kernel<S, CW>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024 - 2048);
        attr = true;
    }
    if (prepare_only) return cudaGetLastError();
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)(g.nsamples * csize));
    cfg.blockDim = dim3(kClusterThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)csize;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, cluster_kernel<S, CW>, p);
}

template <typename S>
cudaError_t launch_cluster_s(const KParams& p, const BatchGeometry& g, cudaStream_t s, bool prepare_only) {
    const int csize = p.cluster_size, cw = p.cluster_cw;
    if (csize < 1 || csize > 16 || cw < 1) return cudaErrorInvalidConfiguration;
    switch (cluster_row_width<S>(cw, p.cluster_ny)) {
        case 16: return launch_cluster_w<S, 16>(p, g, s, prepare_only);
        case 32: return launch_cluster_w<S, 32>(p, g, s, prepare_only);
        case 48: return launch_cluster_w<S, 48>(p, g, s, prepare_only);
        case 64: return launch_cluster_w<S, 64>(p, g, s, prepare_only);
        default: return launch_cluster_w<S, 0>(p, g, s, prepare_only);
    }
}

// Clusters of `csize` blocks with `smem` bytes each that can run at once (0: none).
template <typename S>
int cluster_capacity(int csize, size_t smem) {
    static struct {
        size_t smem;
        int cap;
    } cache[17] = {};
    if (cache[csize].smem == smem && smem != 0) return cache[csize].cap;
    // every row width's kernel runs one 1024-thread block per SM; the 64-column one stands for all
    cudaFuncSetAttribute(cluster_kernel<S, 64>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    cudaFuncSetAttribute(cluster_kernel<S, 64>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024 - 2048);
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)csize);
    cfg.blockDim = dim3(kClusterThreads);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)csize;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, cluster_kernel<S, 64>, &cfg) != cudaSuccess) {
        cudaGetLastError();
        n = 0;
    }
    cache[csize].smem = smem;
    cache[csize].cap = n;
    return n;
}


// ------------------------------------------------------------------------------------------
// Final fields and per-sample scalars at the last step run.
// ------------------------------------------------------------------------------------------
template <typename S, bool MIXED>
__global__ void __launch_bounds__(256) finalize_kernel(KParams p, int64_t total_tiles, int tile_rows, int tile_cols) {
    using C = typename Storage<S>::C;
    constexpr int NT = 256;
    __shared__ double s_red[(NT / 32) * 7];
    __shared__ int s_flag;
    S* arena = static_cast<S*>(p.arena);
    for (int64_t tile = blockIdx.x; tile < total_tiles; tile += gridDim.x) {
        const int j = tile_sample(p, (int)tile, p.nsamples);
        const SampleDev sp = p.samples[j];
        const typename Storage<S>::Q qz = quanta_of<S>(p, j);
        const bool chan = MIXED && sp.kind == UQLB_CASE_CHANNEL;
        const int T = p.steps_run[sp.slot];
        const int lt = (int)tile - sp.tile_base;
        const int y0 = (lt / sp.tiles_x) * tile_rows;
        const uint32_t* mask = (sp.mask_off >= 0) ? p.masks + sp.mask_off : nullptr;
        const InitDev* bz = (chan && sp.bouzidi && mask != nullptr) ? p.init + j : nullptr;
        // two-step scheme: the state is in natural layout on the lattice the last launch wrote
        const bool two = p.sel != nullptr;
        S* lat = arena;
        if (two && on_final_second(p, sp.slot, T)) lat = static_cast<S*>(p.arena2);
        double red[7] = {0, 0, 0, 0, 0, 0, 0};  // K, mass, mx, my, fx, fy, bad
        for (int q = threadIdx.x; q < tile_rows * tile_cols; q += blockDim.x) {
            const int x = (lt % sp.tiles_x) * tile_cols + (q % tile_cols);
            const int y = y0 + q / tile_cols;
            if (x >= sp.nx || y >= sp.ny) continue;
            const bool solid = mask != nullptr && mask_solid(mask, mask_words(sp), x, y);
            double ux = 0.0, uy = 0.0;
            if (!solid) {
                S* base = lat + sp.f_off;
                const int64_t own = (int64_t)y * sp.pitch + x;
                C g[9];
                if constexpr (std::is_same<S, int16_t>::value) {
                    // a value held at the end of the fixed-point range saturated on a store
#pragma unroll
                    for (int i = 0; i < 9; ++i)
                        if (Storage<S>::at_limit(base + i * sp.plane + own)) red[6] += 1.0;
                }
                if (two || p.natural || (T & 1) == 0) {
#pragma unroll
                    for (int i = 0; i < 9; ++i) g[i] = Storage<S>::load(base + i * sp.plane + own, qz, i);
                } else {
                    C ubx = C(0), uby = C(0);
                    if (chan && x == sp.nx - 1) {
                        if (sizeof(C) == 8) {
                            ubx = (C)p.side_d[2 * (sp.side_off + y)];
                            uby = (C)p.side_d[2 * (sp.side_off + y) + 1];
                        } else {
                            ubx = (C)p.side[2 * (sp.side_off + y)];
                            uby = (C)p.side[2 * (sp.side_off + y) + 1];
                        }
                    }
                    g[0] = Storage<S>::load(base + own, qz, 0);
#pragma unroll
                    for (int i = 1; i < 9; ++i)
                        g[i] = read_incoming<S>(base, sp, mask, x, y, i, T - 1, ubx, uby, chan, qz);
                }
                const uint32_t links = bz != nullptr ? obstacle_links(sp, *bz, mask, x, y) : 0u;
                if (links && T > 0) bouzidi_complete(*bz, x, y, links, g);
                if (chan && sp.inout && T > 0 && (x == 0 || x == sp.nx - 1)) {
                    const double* b = p.bcpop + (int64_t)(sp.bc_off + (x == 0 ? 0 : sp.ny) + y) * 9;
#pragma unroll
                    for (int i = 0; i < 9; ++i) g[i] = (C)b[i];
                }
                C drho, cjx, cjy, cux, cuy;
                moments(g, drho, cjx, cjy, cux, cuy);
                ux = (double)cux;
                uy = (double)cuy;
                const double rho = 1.0 + (double)drho;
                red[0] += ux * ux + uy * uy;
                red[1] += rho;
                red[2] += rho * ux;
                red[3] += rho * uy;
                if (!(rho > 0.0) || !isfinite(ux) || !isfinite(uy)) red[6] += 1.0;
                if (mask != nullptr && T > 0) {
                    // halfway: the bounce-back populations at T are the post-collision values of
                    // step T - 1; Bouzidi: c_i (g*_i(T - 1) parked in the obstacle node + the
                    // completed returning population at T)
#pragma unroll
                    for (int i = 1; i < 9; ++i) {
                        const int xn = x + cx(i), yn = y + cy(i);
                        if (xn >= 0 && xn < sp.nx && yn >= 0 && yn < sp.ny &&
                            mask_solid(mask, mask_words(sp), xn, yn)) {
                            if (links) {
                                const double fs =
                                    (double)Storage<S>::load(base + i * sp.plane + (int64_t)yn * sp.pitch + xn, qz, i) +
                                    (double)g[opp(i)] + 2.0 * wgt<double>(i);
                                red[4] += cx(i) * fs;
                                red[5] += cy(i) * fs;
                            } else {
                                const double fs =
                                    (double)Storage<S>::load(base + opp(i) * sp.plane + own, qz, i) + wgt<double>(i);
                                red[4] += 2.0 * cx(i) * fs;
                                red[5] += 2.0 * cy(i) * fs;
                            }
                        }
                    }
                }
            }
            if (p.fields != nullptr) {
                const int64_t row = (int64_t)sp.sample_id * p.fields_ld;
                const int64_t n = (int64_t)sp.nx * sp.ny;
                const int64_t node = (int64_t)y * sp.nx + x;
                if (p.fields_dtype == UQLB_F64) {
                    double* f = static_cast<double*>(p.fields) + row;
                    f[node] = ux;
                    f[n + node] = uy;
                } else {
                    float* f = static_cast<float*>(p.fields) + row;
                    f[node] = (float)ux;
                    f[n + node] = (float)uy;
                }
            }
        }
        double tot[7];
        if (tile_reduce_last<7, NT>(p, sp, j, (int)tile, red, tot, s_red, &s_flag)) {
            if (threadIdx.x == 0) {
                const double K = tot[0] * sp.u_ref_inv2;
                if (p.qoi != nullptr) {
                    double* q = p.qoi + (int64_t)sp.sample_id * UQLB_QOI_COLS;
                    q[UQLB_QOI_K] = K;
                    q[UQLB_QOI_MASS] = tot[1];
                    q[UQLB_QOI_MOMX] = tot[2];
                    q[UQLB_QOI_MOMY] = tot[3];
                    q[UQLB_QOI_CD] = tot[4] * sp.force_norm;
                    q[UQLB_QOI_CL] = tot[5] * sp.force_norm;
                    q[UQLB_QOI_STEPS] = (double)T;
                    q[UQLB_QOI_STATUS] = *(volatile int*)p.bar_err != 0 ? (double)UQLB_ERR_TIMEOUT
                                         : (tot[6] > 0.0 ? (double)UQLB_ERR_UNSTABLE : 0.0);
                }
                if (p.fields != nullptr) {
                    const int64_t at = (int64_t)sp.sample_id * p.fields_ld + 2 * (int64_t)sp.nx * sp.ny;
                    if (p.fields_dtype == UQLB_F64)
                        static_cast<double*>(p.fields)[at] = K;
                    else
                        static_cast<float*>(p.fields)[at] = (float)K;
                }
                if (!chan && p.series != nullptr && p.qoi_every > 0 && T % p.qoi_every == 0)
                    p.series[(int64_t)sp.sample_id * p.series_ld + T / p.qoi_every] = K;
            }
        }
    }
}

// Obstacle force of the Bouzidi samples at time s = step counter + dt + 1 when s is a QoI step:
// F = sum over the obstacle links of c_i (f*_i(x, s-1) + f_ibar(x, s)) (the momentum exchanged on
// the link), from the values the step s-1 left in memory: the parked g*_i, the bounce-back slot
// and, for q < 1/2, the streamed g_i (found as the gather of step s would find it).  One block per
// sample walks the nodes of the obstacle's bounding box.  It runs between the launches of steps
// s-1 and s, so a sample that passes the steady-state test stops with its state at s.
template <typename S>
__global__ void __launch_bounds__(256) bouzidi_force_kernel(KParams p) {
    using C = typename Storage<S>::C;
    constexpr int NT = 256;
    __shared__ double s_red[(NT / 32) * 2];
    const int s = (int)(*p.step_counter) + p.dt + 1;
    if (p.qoi_every <= 0 || s % p.qoi_every != 0) return;
    const bool prev_odd = ((s - 1) & 1) != 0;
    for (int j = blockIdx.x; j < p.nsamples; j += gridDim.x) {
        const SampleDev& sp = p.samples[j];
        if (!sp.bouzidi || sp.mask_off < 0 || s > sp.steps || p.done[sp.slot]) continue;
        const InitDev& in = p.init[j];
        const typename Storage<S>::Q qz = quanta_of<S>(p, j);
        const uint32_t* mask = p.masks + sp.mask_off;
        const S* base = static_cast<const S*>(p.arena) + sp.f_off;
        const int bw = in.bbox[1] - in.bbox[0] + 1, bh = in.bbox[3] - in.bbox[2] + 1;
        const int nbox = (bw > 0 && bh > 0) ? bw * bh : 0;
        double red[2] = {0.0, 0.0};
        for (int n = threadIdx.x; n < nbox; n += NT) {
            const int x = in.bbox[0] + n % bw, y = in.bbox[2] + n / bw;
            if (mask_solid(mask, mask_words(sp), x, y)) continue;
            const uint32_t links = obstacle_links(sp, in, mask, x, y);
            if (!links) continue;
            const int64_t own = (int64_t)y * sp.pitch + x;
            C ubx = C(0), uby = C(0);
            if (prev_odd == false && x == sp.nx - 1) {
                if (sizeof(C) == 8) {
                    ubx = (C)p.side_d[2 * (sp.side_off + y)];
                    uby = (C)p.side_d[2 * (sp.side_off + y) + 1];
                } else {
                    ubx = (C)p.side[2 * (sp.side_off + y)];
                    uby = (C)p.side[2 * (sp.side_off + y) + 1];
                }
            }
#pragma unroll
            for (int i = 1; i < 9; ++i) {
                if (!(links >> i & 1u)) continue;
                C back = Storage<S>::load(base + opp(i) * sp.plane + own, qz, i);
                const C q = link_q<C>(in, x, y, i);
                if (q < C(0.5)) {
                    const C gi = prev_odd ? Storage<S>::load(base + i * sp.plane + own, qz, i)
                                          : read_incoming<S>(base, sp, mask, x, y, i, s - 1, ubx, uby, true, qz);
                    back += (C(1) - C(2) * q) * gi;
                }
                const C parked = Storage<S>::load(base + i * sp.plane + (int64_t)(y + cy(i)) * sp.pitch + (x + cx(i)), qz, i);
                const double fs = (double)parked + (double)back + 2.0 * wgt<double>(i);
                red[0] += cx(i) * fs;
                red[1] += cy(i) * fs;
            }
        }
        block_sum<2, NT>(red, s_red);
        if (threadIdx.x == 0) record_force(p, sp, j, s, red[0], red[1]);
        __syncthreads();
    }
}

// Interpolated inlet/outlet (Sec. 8.1; the finite-difference velocity-gradient conditions of
// Latt et al. 2008): for every sample that uses it and has a state at time s = step counter +
// dt + 1, the populations of its end columns at s, f_i = f_i^eq(rho, u) - 3 w_i rho tau Q_i:S,
// written (shifted, g = f - w) to its boundary buffer, which the step of s and the finalize read
// for those nodes.  Inlet (column 0): u = (parabola at the node centre, 0), rho from the known
// populations; outlet (column nx - 1): rho = 1, u_x from the known populations, u_y that of
// column nx - 2.  The strain rate comes from finite differences: second-order one-sided across
// the column (columns 0, 1, 2 or nx - 1, nx - 2, nx - 3), central along it, one-sided at its
// ends.  The post-stream state of a node is gathered as the step of s would gather it.
template <typename S>
__global__ void __launch_bounds__(256) inout_kernel(KParams p) {
    using C = typename Storage<S>::C;
    const int s = (int)(*p.step_counter) + p.dt + 1;
    for (int j = blockIdx.x; j < p.nsamples; j += gridDim.x) {
        const SampleDev& sp = p.samples[j];
        if (sp.kind != UQLB_CASE_CHANNEL || !sp.inout || s > p.steps_run[sp.slot]) continue;
        const uint32_t* mask = sp.mask_off >= 0 ? p.masks + sp.mask_off : nullptr;
        const S* base = static_cast<const S*>(p.arena) + sp.f_off;
        const typename Storage<S>::Q qz = quanta_of<S>(p, j);
        const int nx = sp.nx, ny = sp.ny;
        // post-stream shifted populations of node (x, yy) at time s
        auto state = [&](int x, int yy, C (&g)[9]) {
            Nbr nb;
            nb.row[1] = yy * sp.pitch;
            if (s & 1)
                node_load<S, true>(p, sp, base, mask, x, yy, s, true, nb, nullptr, 0u, g, qz, false);
            else
                node_load<S, false>(p, sp, base, mask, x, yy, s, true, nb, nullptr, 0u, g, qz, false);
        };
        auto velocity = [&](int x, int yy, C& ux, C& uy) {
            C g[9], drho, jx, jy;
            state(x, yy, g);
            moments(g, drho, jx, jy, ux, uy);
        };
        // outlet node: u_x from its known populations (rho = 1; the known weights sum to 1, so
        // in shifted form u_x = g_0 + g_2 + g_4 + 2 (g_1 + g_5 + g_8)), u_y from column nx - 2
        auto outlet_u = [&](int yy, C& ux, C& uy) {
            C g[9], vx;
            state(nx - 1, yy, g);
            ux = g[0] + g[2] + g[4] + C(2) * (g[1] + g[5] + g[8]);
            velocity(nx - 2, yy, vx, uy);
        };
        const C tau = C(1) / (C)sp.omega;
        for (int y = threadIdx.x; y < ny; y += blockDim.x) {
            for (int side = 0; side < 2; ++side) {
                C u0x, u0y, u1x, u1y, u2x, u2y, drho;
                C ax[3], ay[3];  // boundary-column velocity at the three rows of the y stencil
                const int ys = y == 0 ? 0 : (y == ny - 1 ? ny - 3 : y - 1);
                if (side == 0) {
                    C g[9];
                    state(0, y, g);
                    u0x = inflow<C>(sp, C(y) + C(0.5), s);
                    u0y = C(0);
                    // rho = (1 + G) / (1 - u_x), G the shifted known sum: drho = (G + u_x) / (1 - u_x)
                    const C G = g[0] + g[2] + g[4] + C(2) * (g[3] + g[6] + g[7]);
                    drho = (G + u0x) / (C(1) - u0x);
                    velocity(1, y, u1x, u1y);
                    velocity(2, y, u2x, u2y);
                    for (int k = 0; k < 3; ++k) {
                        ax[k] = inflow<C>(sp, C(ys + k) + C(0.5), s);
                        ay[k] = C(0);
                    }
                } else {
                    outlet_u(y, u0x, u0y);
                    drho = C(0);
                    velocity(nx - 2, y, u1x, u1y);
                    velocity(nx - 3, y, u2x, u2y);
                    for (int k = 0; k < 3; ++k) outlet_u(ys + k, ax[k], ay[k]);
                }
                const C sgn = side == 0 ? C(1) : C(-1);
                const C dxu = sgn * (C(-3) * u0x + C(4) * u1x - u2x) / C(2);
                const C dxv = sgn * (C(-3) * u0y + C(4) * u1y - u2y) / C(2);
                C dyu, dyv;
                if (y == 0) {
                    dyu = (C(-3) * ax[0] + C(4) * ax[1] - ax[2]) / C(2);
                    dyv = (C(-3) * ay[0] + C(4) * ay[1] - ay[2]) / C(2);
                } else if (y == ny - 1) {
                    dyu = (C(3) * ax[2] - C(4) * ax[1] + ax[0]) / C(2);
                    dyv = (C(3) * ay[2] - C(4) * ay[1] + ay[0]) / C(2);
                } else {
                    dyu = (ax[2] - ax[0]) / C(2);
                    dyv = (ay[2] - ay[0]) / C(2);
                }
                const C sxx = dxu, syy = dyv, sxy = C(0.5) * (dyu + dxv);
                const C rho = C(1) + drho, usq = u0x * u0x + u0y * u0y;
                double* b = p.bcpop + (int64_t)(sp.bc_off + side * ny + y) * 9;
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    const C w = wgt<C>(i);
                    const C cu = C(cx(i)) * u0x + C(cy(i)) * u0y;
                    const C q = C(cx(i) * cx(i) - 1.0 / 3.0) * sxx + C(cy(i) * cy(i) - 1.0 / 3.0) * syy +
                                C(2 * cx(i) * cy(i)) * sxy;
                    const C geq = w * drho + w * rho * (C(3) * cu + C(4.5) * cu * cu - C(1.5) * usq);
                    b[i] = (double)(geq - C(3) * w * rho * tau * q);
                }
            }
        }
    }
}

// Resident blocks per SM of one step-kernel instantiation (queried once).
template <typename S, bool ODD, bool MIXED, int TR, int NPT>
int resident_blocks() {
    static int n = 0;
    if (n == 0) {
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, step_kernel<S, ODD, MIXED, TR, NPT>, kTileCols * TR, 0) !=
                cudaSuccess || b < 1)
            b = 1;
        n = b;
    }
    return n;
}

template <typename S, bool ODD, bool MIXED, int TR, int NPT>
cudaError_t launch_geom(const KParams& p, const BatchGeometry& g, cudaStream_t s) {
    const int64_t resident = (int64_t)resident_blocks<S, ODD, MIXED, TR, NPT>() * sm_count();
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(g.total_tiles, resident));
    step_kernel<S, ODD, MIXED, TR, NPT><<<grid, dim3(kTileCols, TR), 0, s>>>(p);
    return cudaGetLastError();
}

// Geometries compiled for each (storage, mixed) combination; see geometry_supported().
#define UQLB_GEOM(TR_, NPT_) \
    if (g.tile_rows == TR_ && g.npt == NPT_) return launch_geom<S, ODD, MIXED, TR_, NPT_>(p, g, s);
template <typename S, bool ODD, bool MIXED>
cudaError_t launch_step_geom(const KParams& p, const BatchGeometry& g, cudaStream_t s) {
    if constexpr (MIXED) {
        UQLB_GEOM(8, 1)
        UQLB_GEOM(4, 1)
    } else if constexpr (sizeof(S) == 8) {
        UQLB_GEOM(8, 1)
        UQLB_GEOM(4, 1)
        UQLB_GEOM(4, 2)
    } else {
        UQLB_GEOM(2, 1)
        UQLB_GEOM(4, 1)
        UQLB_GEOM(8, 1)
        UQLB_GEOM(2, 2)
        UQLB_GEOM(4, 2)
        UQLB_GEOM(8, 2)
        UQLB_GEOM(2, 4)
        UQLB_GEOM(4, 4)
        UQLB_GEOM(8, 4)
    }
    return cudaErrorInvalidConfiguration;
}
#undef UQLB_GEOM

template <typename S>
cudaError_t launch_step_s(const KParams& p, const BatchGeometry& g, bool odd, cudaStream_t s) {
    if (g.any_channel)
        return odd ? launch_step_geom<S, true, true>(p, g, s) : launch_step_geom<S, false, true>(p, g, s);
    return odd ? launch_step_geom<S, true, false>(p, g, s) : launch_step_geom<S, false, false>(p, g, s);
}


template <typename S, int TR, int NPT>
constexpr size_t step2_smem() {
    return sizeof(typename Storage<S>::C) * 9 * (TR + 2) * (kTileCols * NPT + 2);
}

// Shared-memory opt-in and resident blocks per SM of one two-step instantiation (once).
template <typename S, int TR, int NPT>
int resident_blocks2() {
    static int n = 0;
    if (n == 0) {
        constexpr size_t smem = step2_smem<S, TR, NPT>();
        cudaFuncSetAttribute(step2_kernel<S, TR, NPT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, step2_kernel<S, TR, NPT>, kTileCols * TR, smem) !=
                cudaSuccess || b < 1)
            b = 1;
        n = b;
    }
    return n;
}

template <typename S, int TR, int NPT>
cudaError_t launch_geom2(const KParams& p, const BatchGeometry& g, cudaStream_t s, bool prepare_only) {
    const int64_t resident = (int64_t)resident_blocks2<S, TR, NPT>() * sm_count();
    if (prepare_only) return cudaGetLastError();
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(g.total_tiles, resident));
    step2_kernel<S, TR, NPT><<<grid, dim3(kTileCols, TR), step2_smem<S, TR, NPT>(), s>>>(p);
    return cudaGetLastError();
}

#define UQLB_GEOM2(TR_, NPT_) \
    if (g.tile_rows == TR_ && g.npt == NPT_) return launch_geom2<S, TR_, NPT_>(p, g, s, prepare_only);
template <typename S>
cudaError_t launch_step2_s(const KParams& p, const BatchGeometry& g, cudaStream_t s, bool prepare_only) {
    if constexpr (sizeof(S) == 8) {
        UQLB_GEOM2(4, 2)
        UQLB_GEOM2(8, 1)
        UQLB_GEOM2(8, 2)
    } else {
        UQLB_GEOM2(4, 4)
        UQLB_GEOM2(8, 2)
        UQLB_GEOM2(8, 4)
        UQLB_GEOM2(16, 2)
        UQLB_GEOM2(16, 4)
    }
    return cudaErrorInvalidConfiguration;
}
#undef UQLB_GEOM2

template <typename S>
size_t strip_smem(int nx) {
    return (size_t)kStripPlanes * nx * sizeof(float) + (size_t)StripTune<S>::depth * 9 * nx * sizeof(S);
}

// Shared-memory opt-in (for the widest rows) and resident blocks per SM at width nx (once each).
template <typename S, bool GENERIC>
int strip_resident(int nx) {
    constexpr int kb = StripTune<S>::carveout_kb;
    const int np = strip_threads(nx), rw = 2 * np;
    static int cache[1024 / 32 + 1] = {};
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(strip2_kernel<S, GENERIC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)strip_smem<S>(StripTune<S>::max_nx));
        // percent of the 228 KB maximum, rounded down: the driver rounds up to the next supported split
        if (kb > 0) cudaFuncSetAttribute(strip2_kernel<S, GENERIC>, cudaFuncAttributePreferredSharedMemoryCarveout, kb * 100 / 228);
        attr = true;
    }
    int& n = cache[np / 32];
    if (n == 0) {
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, strip2_kernel<S, GENERIC>, np, strip_smem<S>(rw)) != cudaSuccess ||
            b < 1)
            b = 1;
        if (kb > 0) {
            // blocks that fit the preferred share (each with its static part and 1 KB reserve), so
            // that the grid stays resident in one wave
            cudaFuncAttributes fa{};
            cudaFuncGetAttributes(&fa, strip2_kernel<S, GENERIC>);
            const size_t per = strip_smem<S>(rw) + fa.sharedSizeBytes + 1024;
            b = std::max(1, std::min(b, (int)((size_t)kb * 1024 / per)));
        }
        n = b;
    }
    return n;
}

template <typename S>
cudaError_t launch_strip_s(const KParams& p, const BatchGeometry& g, cudaStream_t s, bool prepare_only) {
    const int np = strip_threads(g.strip_nx);
    if (g.strip_nx < 2 || 2 * np > StripTune<S>::max_nx) return cudaErrorInvalidConfiguration;
    const bool generic = g.strip_nx != 2 * np;
    const int64_t resident =
        (int64_t)(generic ? strip_resident<S, true>(g.strip_nx) : strip_resident<S, false>(g.strip_nx)) * sm_count();
    if (prepare_only) return cudaGetLastError();
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(g.total_rows, resident));
    if (generic)
        strip2_kernel<S, true><<<grid, np, strip_smem<S>(2 * np), s>>>(p);
    else
        strip2_kernel<S, false><<<grid, np, strip_smem<S>(2 * np), s>>>(p);
    return cudaGetLastError();
}


template <typename S, bool MIXED, int TR, int NPT>
cudaError_t launch_persistent_geom(const KParams& p, int chunk, cudaStream_t s) {
    static int per_sm = 0;
    if (per_sm == 0) {
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, persistent_kernel<S, MIXED, TR, NPT>, kTileCols * TR, 0) !=
                cudaSuccess || b < 1)
            b = 1;
        per_sm = b;
    }
    const int grid = per_sm * sm_count();
    KParams pp = p;
    int ch = chunk;
    void* args[] = {&pp, &ch};
    return cudaLaunchCooperativeKernel((const void*)persistent_kernel<S, MIXED, TR, NPT>, dim3(grid),
                                       dim3(kTileCols, TR), args, 0, s);
}

#define UQLB_PGEOM(TR_, NPT_) \
    if (g.tile_rows == TR_ && g.npt == NPT_) return launch_persistent_geom<S, MIXED, TR_, NPT_>(p, chunk, s);
template <typename S, bool MIXED>
cudaError_t launch_persistent_s(const KParams& p, const BatchGeometry& g, int chunk, cudaStream_t s) {
    if constexpr (MIXED) {
        UQLB_PGEOM(8, 1)
        UQLB_PGEOM(4, 1)
    } else if constexpr (sizeof(S) == 8) {
        UQLB_PGEOM(8, 1)
        UQLB_PGEOM(4, 1)
        UQLB_PGEOM(4, 2)
    } else {
        UQLB_PGEOM(2, 1)
        UQLB_PGEOM(4, 1)
        UQLB_PGEOM(8, 1)
        UQLB_PGEOM(2, 2)
        UQLB_PGEOM(4, 2)
        UQLB_PGEOM(8, 2)
        UQLB_PGEOM(2, 4)
        UQLB_PGEOM(4, 4)
        UQLB_PGEOM(8, 4)
    }
    return cudaErrorInvalidConfiguration;
}
#undef UQLB_PGEOM


// Launchers of the kernels that the dispatcher does not shape itself (grid from the tile count).
inline int64_t tile_grid(const BatchGeometry& g) {
    int64_t grid = g.total_tiles < 65535 * 4 ? g.total_tiles : 65535 * 4;
    return grid < 1 ? 1 : grid;
}

template <typename S>
cudaError_t launch_init_s(const KParams& p, const BatchGeometry& g, cudaStream_t s) {
    init_kernel<S><<<(int)tile_grid(g), 256, 0, s>>>(p, g.total_tiles, g.tile_rows, 32 * g.npt);
    return cudaGetLastError();
}

template <typename S>
cudaError_t launch_finalize_s(const KParams& p, const BatchGeometry& g, cudaStream_t s) {
    if (g.any_channel)
        finalize_kernel<S, true><<<(int)tile_grid(g), 256, 0, s>>>(p, g.total_tiles, g.tile_rows, 32 * g.npt);
    else
        finalize_kernel<S, false><<<(int)tile_grid(g), 256, 0, s>>>(p, g.total_tiles, g.tile_rows, 32 * g.npt);
    return cudaGetLastError();
}

template <typename S>
cudaError_t launch_inout_s(const KParams& p, const BatchGeometry& g, cudaStream_t s) {
    inout_kernel<S><<<(int)(g.nsamples < 4096 ? g.nsamples : 4096), 256, 0, s>>>(p);
    return cudaGetLastError();
}

template <typename S>
cudaError_t launch_bouzidi_force_s(const KParams& p, const BatchGeometry& g, cudaStream_t s) {
    bouzidi_force_kernel<S><<<(int)(g.nsamples < 4096 ? g.nsamples : 4096), 256, 0, s>>>(p);
    return cudaGetLastError();
}

template <typename S>
size_t strip3_smem(int nx) {
    return (size_t)2 * kRing3Planes * nx * sizeof(float) + (size_t)Strip3Tune<S>::depth * 9 * nx * sizeof(S);
}

// Carveout (percent of the largest share) that selects configuration `kb`: rounded down, since the
// driver rounds the share up to the next configuration.
inline int carveout_pct(int kb) { return kb * 100 / 228; }

// Resident blocks per SM and shared-memory share of a row-strip launch: the blocks per SM asked for
// (g.strip_bps, else the default, never above what fits) and the share (g.strip_smem_kb, else the
// default; never below what the blocks need).
inline void strip_launch_shape(const StripBlocks& sb, const BatchGeometry& g, int* bps, int* kb) {
    int b = g.strip_bps > 0 ? std::min(g.strip_bps, sb.max_b) : sb.def_b;
    int k = g.strip_smem_kb > 0 ? g.strip_smem_kb : sb.def_kb;
    k = std::max(k, smem_config_for((size_t)b * sb.per_block));
    *bps = b;
    *kb = k;
}

// Launch of a row-strip kernel over min(total rows, bps x SMs) blocks with the shared-memory share
// as a launch attribute (it holds for this launch only, also inside a captured graph).
template <typename K>
cudaError_t launch_strip_kernel(K kernel, const StripBlocks& sb, const BatchGeometry& g, int threads, size_t smem,
                                const KParams& p, cudaStream_t s) {
    int bps = 0, kb = 0;
    strip_launch_shape(sb, g, &bps, &kb);
    const int64_t resident = (int64_t)bps * sm_count();
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)std::max<int64_t>(1, std::min<int64_t>(g.total_rows, resident)));
    cfg.blockDim = dim3((unsigned)threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributePreferredSharedMemoryCarveout;
    at[0].val.sharedMemCarveout = (unsigned)carveout_pct(kb);
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, p);
}

// Blocks per SM of a kernel with `dyn` bytes of dynamic shared memory at `threads` threads: the
// most that fit (registers and the largest share) and the default under the compiled share.
template <typename K>
StripBlocks strip_blocks_of(K kernel, int threads, size_t dyn, int default_kb) {
    StripBlocks r{};
    cudaFuncAttributes fa{};
    cudaFuncGetAttributes(&fa, kernel);
    r.per_block = (int)(dyn + fa.sharedSizeBytes + 1024);  // 1 KB per block is reserved by the system
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel, threads, dyn) != cudaSuccess || b < 1) b = 1;
    r.max_b = b;
    r.def_b = default_kb > 0 ? std::max(1, std::min(b, default_kb * 1024 / r.per_block)) : b;
    // default_kb: the compiled share; 0: the largest; -1: the smallest holding the blocks
    r.def_kb = default_kb > 0 ? default_kb : (default_kb < 0 ? smem_config_for((size_t)b * r.per_block) : 228);
    return r;
}

// Blocks per SM of the three-step strips at width nx (once per width).
template <typename S, bool GENERIC>
const StripBlocks& strip3_generic_blocks(int nx) {
    const int np = strip_threads(nx), rw = 2 * np;
    static StripBlocks cache[1024 / 32 + 1] = {};
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(strip3_kernel<S, GENERIC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)strip3_smem<S>(Strip3Tune<S>::max_nx));
        attr = true;
    }
    StripBlocks& b = cache[np / 32];
    if (b.max_b == 0) b = strip_blocks_of(strip3_kernel<S, GENERIC>, np, strip3_smem<S>(rw), Strip3Tune<S>::carveout_kb);
    return b;
}

template <typename S, int W, int D>
size_t strip3w_smem() {
    return (size_t)2 * kRing3Planes * (W + 4) * sizeof(float) + (size_t)(D == 1 ? 1 : 0) * 9 * W * sizeof(S);
}

// Blocks per SM of the fixed-width three-step strips (once).
template <typename S, int W, int D>
const StripBlocks& strip3w_blocks() {
    static const StripBlocks b = [] {
        cudaFuncSetAttribute(strip3w_kernel<S, W, D>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)strip3w_smem<S, W, D>());
        // register staging: by default the most blocks that fit and the smallest share that holds
        // them (the rest of the 256 KB as L1: FP32 4 blocks and 164 KB, 0.170 against 0.202 ms per
        // step at 228 KB)
        return strip_blocks_of(strip3w_kernel<S, W, D>, W / 2, strip3w_smem<S, W, D>(),
                               D == 2 ? -1 : Strip3Tune<S>::carveout_kb);
    }();
    return b;
}

// Staging of a fixed-width launch's phase-A rows: option 1 = none, 2 = the next row in shared memory
// by cp.async, 3 = the next row in registers (0: the compiled default); as the kernel's D: 0, 1, 2.
// The default is register staging (measured on the 625 x 256^2 ensemble, kernel GLUPS, none / shared
// memory / registers: FP32 199 / 228 / 241, BF16 219 / 227 / 234, FP16 214 / 223 / 230, FX16 200 / 204
// / 216; `def`, the runtime-width kernel's compiled staging, is not used).
inline int strip3w_depth(int stage, int def) {
    (void)def;
    return stage == 1 ? 0 : (stage == 2 ? 1 : 2);
}

template <typename S, int W, int D>
cudaError_t launch_strip3w_d(const KParams& p, const BatchGeometry& g, cudaStream_t s, bool prepare_only) {
    const StripBlocks& sb = strip3w_blocks<S, W, D>();
    if (prepare_only) return cudaGetLastError();
    return launch_strip_kernel(strip3w_kernel<S, W, D>, sb, g, W / 2, strip3w_smem<S, W, D>(), p, s);
}

template <typename S, int W>
cudaError_t launch_strip3w(const KParams& p, const BatchGeometry& g, cudaStream_t s, bool prepare_only) {
    switch (strip3w_depth(g.strip_stage, Strip3Tune<S>::depth)) {
        case 0: return launch_strip3w_d<S, W, 0>(p, g, s, prepare_only);
        case 1: return launch_strip3w_d<S, W, 1>(p, g, s, prepare_only);
        default: return launch_strip3w_d<S, W, 2>(p, g, s, prepare_only);
    }
}

template <typename S, int W>
const StripBlocks& strip3w_blocks_at(int d) {
    return d == 0 ? strip3w_blocks<S, W, 0>() : (d == 1 ? strip3w_blocks<S, W, 1>() : strip3w_blocks<S, W, 2>());
}

template <typename S>
cudaError_t launch_strip3_s(const KParams& p, const BatchGeometry& g, cudaStream_t s, bool prepare_only) {
    const int np = strip_threads(g.strip_nx);
    if (g.strip_nx < 2 || 2 * np > Strip3Tune<S>::max_nx) return cudaErrorInvalidConfiguration;
    const bool generic = g.strip_nx != 2 * np;
    if (strip3_fixed_width(g.strip_nx)) {
        // the widths with a compile-time instantiation (immediate addressing)
        switch (g.strip_nx) {
            case 64: return launch_strip3w<S, 64>(p, g, s, prepare_only);
            case 128: return launch_strip3w<S, 128>(p, g, s, prepare_only);
            case 256: return launch_strip3w<S, 256>(p, g, s, prepare_only);
            case 512: return launch_strip3w<S, 512>(p, g, s, prepare_only);
            default: return launch_strip3w<S, 1024>(p, g, s, prepare_only);
        }
    }
    const StripBlocks& sb =
        generic ? strip3_generic_blocks<S, true>(g.strip_nx) : strip3_generic_blocks<S, false>(g.strip_nx);
    if (prepare_only) return cudaGetLastError();
    if (generic) return launch_strip_kernel(strip3_kernel<S, true>, sb, g, np, strip3_smem<S>(2 * np), p, s);
    return launch_strip_kernel(strip3_kernel<S, false>, sb, g, np, strip3_smem<S>(2 * np), p, s);
}

// Blocks per SM of the three-step strips of batch g at staging option `stage` (fixed widths only;
// 0: the default).
template <typename S>
bool strip3_blocks_s(const BatchGeometry& g, int stage, StripBlocks* out) {
    if constexpr (sizeof(S) == 8) {
        return false;
    } else {
        const int np = strip_threads(g.strip_nx);
        if (!g.strips || g.spl != 3 || g.strip_nx < 2 || 2 * np > Strip3Tune<S>::max_nx) return false;
        if (strip3_fixed_width(g.strip_nx)) {
            const int d = strip3w_depth(stage, Strip3Tune<S>::depth);
            switch (g.strip_nx) {
                case 64: *out = strip3w_blocks_at<S, 64>(d); break;
                case 128: *out = strip3w_blocks_at<S, 128>(d); break;
                case 256: *out = strip3w_blocks_at<S, 256>(d); break;
                case 512: *out = strip3w_blocks_at<S, 512>(d); break;
                default: *out = strip3w_blocks_at<S, 1024>(d); break;
            }
            return true;
        }
        if (stage != 0) return false;
        *out = g.strip_nx != 2 * np ? strip3_generic_blocks<S, true>(g.strip_nx)
                                     : strip3_generic_blocks<S, false>(g.strip_nx);
        return true;
    }
}

template <typename S>
cudaError_t launch_two_step_s(const KParams& p, const BatchGeometry& g, cudaStream_t s, bool prepare_only) {
    if (g.strips) {
        if constexpr (sizeof(S) == 8) return cudaErrorInvalidConfiguration;
        else if (g.spl == 3) return launch_strip3_s<S>(p, g, s, prepare_only);
        else return launch_strip_s<S>(p, g, s, prepare_only);
    }
    return launch_step2_s<S>(p, g, s, prepare_only);
}

template <typename S>
cudaError_t launch_persistent_any(const KParams& p, const BatchGeometry& g, int chunk, cudaStream_t s) {
    return g.any_channel ? launch_persistent_s<S, true>(p, g, chunk, s) : launch_persistent_s<S, false>(p, g, chunk, s);
}

template <typename S>
cudaError_t launch_cluster_any(const KParams& p, const BatchGeometry& g, cudaStream_t s, bool prepare_only) {
    if constexpr (sizeof(S) == 8) {
        return cudaErrorInvalidConfiguration;  // FP64 lattices do not fit a cluster's shared memory
    } else {
        // cluster size: every size of 1..16 whose blocks hold the widest sample's slab; among them the
        // one with the least estimated time, waves of clusters (the samples over the clusters that
        // run at once) x the time of a step, which is latency-bound: about that of kClusterStepFixed
        // node updates plus one per node of a block's slab (measured on 220 x 41 to 440 x 82
        // channels: 3.3 us + 1 ns per node of the slab).  Larger clusters on ties.
        KParams q = p;
        int best_c = 0, best_cw = 0;
        double best_cost = 0.0;
        for (int c = 16; c >= 1; --c) {
            const int cw = (g.cluster_nx + c - 1) / c, w = cluster_row_width<S>(cw, g.cluster_ny);
            const size_t smem = cluster_smem<S>(w, cw, g.cluster_ny);
            if (smem > kClusterSmemMax) continue;
            const int cap = cluster_capacity<S>(c, smem);
            if (cap < 1) continue;
            const double waves = (double)((g.nsamples + cap - 1) / cap);
            const double cost = waves * (kClusterStepFixed + (double)cw * g.cluster_ny);
            if (best_c == 0 || cost < best_cost) {
                best_cost = cost;
                best_c = c;
                best_cw = cw;
            }
        }
        if (best_c == 0) return cudaErrorInvalidConfiguration;
        g_cluster_choice[0] = best_c;
        g_cluster_choice[1] = best_cw;
        q.cluster_size = best_c;
        q.cluster_cw = best_cw;
        q.cluster_ny = g.cluster_ny;
        return launch_cluster_s<S>(q, g, s, prepare_only);
    }
}

template <typename S>
StorageOps make_storage_ops() {
    StorageOps o;
    o.init = launch_init_s<S>;
    o.step = launch_step_s<S>;
    o.two_step = launch_two_step_s<S>;
    o.persistent = launch_persistent_any<S>;
    o.finalize = launch_finalize_s<S>;
    o.inout = launch_inout_s<S>;
    o.bouzidi_force = launch_bouzidi_force_s<S>;
    o.cluster = launch_cluster_any<S>;
    o.strip3_blocks = strip3_blocks_s<S>;
    return o;
}

}  // namespace

}  // namespace uqlb
