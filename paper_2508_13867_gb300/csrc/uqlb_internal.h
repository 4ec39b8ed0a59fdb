// Internal declarations shared by the host code (uqlb_host.cpp) and the CUDA launchers.
// Not part of the public ABI (include/uqlb.h).
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

#include "../../include/uqlb.h"

namespace uqlb {

// Per-sample parameters as the step kernels read them.  One 128-byte record per sample;
// records are ordered by descending step count so that the samples still running at step t
// form a prefix of the table.
struct alignas(16) SampleDev {
    int64_t f_off;      // element offset of the sample's populations in the arena
    int64_t plane;      // element stride between populations: cols * ny (one-step runs) or cols
                        // (multi-step runs, whose rows keep their nine populations together)
    int32_t nx, ny;
    int32_t pitch;      // element stride between rows: cols (one-step) or 9 cols (multi-step); cols = nx
                        // rounded up to 128 bytes
    int32_t kind;       // UQLB_CASE_TGV / UQLB_CASE_CHANNEL
    int32_t steps;      // steps to run (TGV) or step cap (CHANNEL)
    int32_t sample_id;  // row of the sample in the caller's outputs
    int32_t tiles_x;    // tiles per tile row
    int32_t tiles;      // tiles of this sample
    int32_t tile_base;  // index of the first tile of this sample in the global tile order
    int32_t mask_off;   // word offset of the obstacle bitmask (-1: no obstacle)
    int32_t slot;       // position in the caller's list: the sample's lattice region and the index
                        // of its state that outlives a run (done, steps_run, sel, cd_prev, streak)
    int32_t side_off;   // offset (in pairs) of the outlet velocity buffer
    double omega;       // 1 / tau
    double u_ref_inv2;  // 2 / (nx ny u_ref^2), 0 when K is disabled
    double uin_max;     // channel: peak inflow velocity (1.5 x mean)
    double force_norm;  // channel: 2 / (rho0 u_mean^2 D)
    double ramp_steps;  // channel: ramp length (0: none)
    double steady_tol;  // channel: steady-state tolerance (0: none)
    int32_t steady_checks;  // channel: consecutive passing checks needed (>= 1)
    int32_t bouzidi;        // channel: 1 = Bouzidi interpolated bounce-back on the obstacle
    int32_t inout;          // channel: 1 = interpolated inlet/outlet on the end columns
    int32_t bc_off;         // channel with inout: first node of its boundary buffer (2 x ny nodes)
};
static_assert(sizeof(SampleDev) == 128, "SampleDev must stay 128 bytes");
// 32-bit words per obstacle-mask row.
__host__ __device__ inline int mask_words(const SampleDev& s) { return (s.nx + 31) >> 5; }

// Initial-field parameters (read by the init kernel) and the obstacle geometry (read by the
// Bouzidi links, which are rare: only nodes inside bbox look at it).
struct alignas(16) InitDev {
    double u0, amp2, amp3;
    double pad;
    double pert[4];  // perturbed TGV amplitudes zeta_00, zeta_01, zeta_10, zeta_11
    double cyl_cx, cyl_cy, cyl_r;
    double pad2;
    int32_t bbox[4];  // x0, x1, y0, y1 (inclusive): the only nodes that can have obstacle links
    // 16-bit fixed-point storage: quantum of the rest, axis and diagonal populations and its inverse
    float quanta[4];
    float inv_quanta[4];
};

// Device pointers carved out of the caller's workspace for one batch run.
struct BatchBuffers {
    void* arena;             // populations, storage type
    void* arena2;            // second lattice of the two-step scheme (nullptr: one-step scheme)
    int32_t* sel;            // [S] two-step scheme: lattice (0/1) holding the state at the run's start
    int32_t* row_base;       // [S + 1] first row of each sample in table order (row-strip kernel)
    SampleDev* samples;      // [S] ordered by descending steps
    InitDev* init;           // [S] same order
    int32_t* steps_sorted;   // [S] descending
    uint32_t* masks;         // obstacle bitmasks
    float* side;             // outlet velocities (float pairs)
    double* side_d;          // outlet velocities (double pairs, FP64 storage)
    double* bcpop;           // interpolated inlet/outlet: next state of the end columns, 9 per node
    double* partials;        // [tiles x 3] per-tile QoI partial sums
    int32_t* counters;       // [S] tiles finished in the current reduction
    int32_t* done;           // [S] 1 once a sample has stopped (steady state)
    int32_t* steps_run;      // [S]
    double* cd_prev;         // [S] previous C_D check
    int32_t* streak;         // [S] consecutive passing steady-state checks
    unsigned int* bar_count; // persistent mode: grid barrier arrivals
    unsigned int* bar_gen;   //   and generation
    int32_t* bar_err;        //   nonzero once a bounded wait gave up (UQLB_ERR_TIMEOUT)
    unsigned long long* tickets;  // persistent mode: tile ticket counter of the running chunk
    int64_t* step_counter;   // [2] base step of the running graph chunk, first step of the run
    int32_t* active_flag;    // [1] nonzero while any channel sample still runs
};

struct BatchGeometry {
    int64_t nsamples;
    int64_t total_tiles;
    int64_t total_rows;      // rows of all samples (row-strip kernel)
    int32_t tile_rows;       // rows per tile (threads per block = 32 x tile_rows)
    int32_t npt;             // nodes per thread along x (tile width 32 x npt)
    int32_t max_steps;
    int32_t storage;
    int32_t any_channel;
    int32_t uniform_tiles;   // tiles per sample when every sample has the same size, else 0
    int32_t stochastic;      // 16-bit storage rounds stochastically
    int32_t test_withhold;   // persistent mode test hook: block 0 withholds its barrier arrival
    int32_t any_bouzidi;     // some sample uses the Bouzidi obstacle scheme
    int32_t two_step;        // UQLB_SCHEME_TWO_STEP: one launch per two steps on two lattices
    int32_t any_inout;       // some sample uses the interpolated inlet/outlet
    int32_t strips;          // two-step scheme on row strips (strip2_kernel) instead of tiles
    int32_t strip_nx;        // width of every sample when strips is set
    int32_t spl;             // time steps per launch: 1 (one-step), 2 (tiles, two-step strips), 3 (three-step strips)
    int32_t cluster;         // UQLB_SCHEME_CLUSTER: one thread-block cluster per sample holds it on chip
    int32_t cluster_nx, cluster_ny;  // cluster runs: largest sample width and height
    int32_t strip_bps;       // three-step strips: resident blocks per SM (0: default)
    int32_t strip_stage;     // three-step strips at fixed widths: 1 = no staged row, 2 = one (0: default)
    int32_t strip_smem_kb;   // three-step strips: shared-memory share per SM in KB (0: default)
    int32_t pad_;            // keeps the struct free of padding bytes (it keys the graph cache)
};

// Output pointers of a run (rows indexed by SampleDev::sample_id).
struct RunOutputs {
    void* fields;
    int64_t fields_ld;
    int32_t fields_dtype;
    double* qoi;
    double* series;
    double* series_cl;
    int64_t series_ld;
    int64_t qoi_every;
};

// Launchers (lbm_launch.cu; kernels in lbm_kernels.cuh, one translation unit per storage type).
cudaError_t launch_init(const BatchBuffers& b, const BatchGeometry& g, cudaStream_t s);
// Step dt of a chunk whose base step has parity base_parity (the AA parity of the launch).
cudaError_t launch_step(const BatchBuffers& b, const BatchGeometry& g, const RunOutputs& o,
                        int dt, int base_parity, cudaStream_t s);
// Obstacle force of the Bouzidi samples at step dt + 1 of a chunk (no-op off the QoI steps);
// launched after step dt of the chunk, before step dt + 1.
cudaError_t launch_bouzidi_force(const BatchBuffers& b, const BatchGeometry& g, const RunOutputs& o,
                                 int dt, int base_parity, cudaStream_t s);
cudaError_t launch_advance(const BatchBuffers& b, int chunk, cudaStream_t s);
// Interpolated inlet/outlet: the end-column state at step dt + 1 of a chunk into the boundary
// buffer; launched after step dt of the chunk, before step dt + 1.
cudaError_t launch_inout(const BatchBuffers& b, const BatchGeometry& g, int dt, cudaStream_t s);
// Two-step scheme: steps dt and dt + 1 of a chunk in one launch (one step for samples that end at
// dt + 1); commit: after finalize, record which lattice holds each sample's final state.
cudaError_t launch_step2(const BatchBuffers& b, const BatchGeometry& g, const RunOutputs& o, int dt,
                         cudaStream_t s);
cudaError_t launch_commit(const BatchBuffers& b, const BatchGeometry& g, cudaStream_t s);
// Shared-memory opt-in of the two-step kernel of g's geometry; call before capturing a graph.
cudaError_t prepare_step2(const BatchGeometry& g);
cudaError_t launch_resume(const BatchBuffers& b, const BatchGeometry& g, cudaStream_t s);
// Persistent mode: one cooperative launch runs `chunk` steps (tile tickets must be zero).
cudaError_t launch_persistent(const BatchBuffers& b, const BatchGeometry& g, const RunOutputs& o, int chunk,
                              cudaStream_t s);
cudaError_t launch_finalize(const BatchBuffers& b, const BatchGeometry& g, const RunOutputs& o,
                            cudaStream_t s);
// Blocks per cluster and columns per block the last cluster launch chose.
void last_cluster_choice(int* blocks, int* cols);
// Cluster runs: every sample's whole time loop on chip in one launch.
cudaError_t launch_cluster(const BatchBuffers& b, const BatchGeometry& g, const RunOutputs& o, cudaStream_t s);
bool geometry_supported(int storage, bool mixed, int tile_rows, int npt);
bool geometry_supported2(int storage, int tile_rows, int npt);  // two-step scheme
// Row-strip two-step kernel: FP32/FP16/BF16 storage, sample width a multiple of 64 in 64..2048.
bool strip_supported(int storage, int nx);
// Three-step row strips: FP32 rows up to 1280 wide, 16-bit up to 1600 (rounded up to 64 columns).
bool strip3_supported(int storage, int nx);
// Whether a cluster run holds a channel sample of nx x ny nodes (its lattice once in the shared
// memory of at most 16 blocks, with the link words and the node lists); host arithmetic only.
bool cluster_fits(int storage, int nx, int ny);
// Widths of the three-step strips with a compile-time instantiation (immediate addressing, and a
// staging option per launch).
#ifndef UQLB_STRIP3_FIXED_WIDTHS
#define UQLB_STRIP3_FIXED_WIDTHS 1
#endif
// Shared-memory configurations per SM (KB) that a carveout selects (the rest of the 256 KB is L1),
// and the smallest one holding `bytes`.
constexpr int kSmemConfigsKB[] = {0, 8, 16, 32, 64, 100, 132, 164, 196, 228};
inline int smem_config_for(size_t bytes) {
    for (int kb : kSmemConfigsKB)
        if ((size_t)kb * 1024 >= bytes) return kb;
    return 228;
}
inline bool strip3_fixed_width(int nx) {
    return UQLB_STRIP3_FIXED_WIDTHS && (nx == 64 || nx == 128 || nx == 256 || nx == 512 || nx == 1024);
}
// Three-step strips of batch g at staging option `stage` (1: none, 2: one row, 0: default): the
// most resident blocks per SM, the default, the default shared-memory share (KB) and the shared
// memory per block (bytes).  False when g does not run on the three-step strips or the staging
// option does not apply to its width.
bool strip3_blocks(const BatchGeometry& g, int stage, int* max_b, int* def_b, int* def_kb, int* per_block);

// Plain per-sample FP64 path (plain_f64.cu).
struct PlainSample {
    int32_t nx, ny, kind, steps;
    double omega, u0, amp2, amp3, u_ref_inv2, uin_max, force_norm, ramp_steps;
    double cyl_cx, cyl_cy, cyl_r;
};
cudaError_t plain_run_sample(const PlainSample& p, double* f_a, double* f_b, uint8_t* solid,
                             double* partials, int64_t qoi_every, double* fields,
                             double* qoi_row, double* series_row, cudaStream_t s);

// Wasserstein-1 of speed distributions (w1_kernels.cu); ws holds 256 + 2 * bins * 4 bytes,
// out_dev four doubles (distance, bin width, non-finite speeds of set a and of set b).
cudaError_t launch_w1_speed(const void* a, int dta, int64_t sa, int64_t na, int64_t lda, const void* b, int dtb,
                            int64_t sb, int64_t nb, int64_t ldb, int bins, void* ws, double* out_dev, cudaStream_t s);

// Context accessors for entry points implemented outside uqlb_host.cpp.
int ctx_projection_view(uqlb_ctx* ctx, const double** W, int* K, int64_t* S, int* device);
int ctx_fail(uqlb_ctx* ctx, int code, const char* msg);

// Postprocessing (project_kernels.cu).
// Points per dimension and polynomial degree up to which the projection on a tensor Gauss-Legendre
// grid is sum-factorized.
constexpr int kSfMaxPoints = 16;
constexpr int kSfMaxDegree = 8;
// One stage of the sum-factorized projection (project_kernels.cu): out[r jout + oidx[j' p1 + a]][f] =
// sum_{q < n} G[a n + q] in[(r n + q) jprev + j'][f] over groups (r, j'), rows of stride in_ld / out_ld.
cudaError_t launch_sf_stage(const void* in, int in_dtype, int64_t in_ld, double* out, int64_t out_ld, int64_t groups,
                            int jprev, int jout, int n, int p1, const int* oidx, const double* G, int64_t F,
                            cudaStream_t s);
cudaError_t launch_project(const double* W, int K, int S, const void* M, int dtype,
                           int64_t F, int64_t ld, double* C, cudaStream_t s);
cudaError_t launch_gpc_stats(const double* C, int K, int64_t F, double* mean, double* var,
                             cudaStream_t s);
cudaError_t launch_mc_stats(const void* M, int dtype, int64_t S, int64_t F, int64_t ld,
                            double* mean, double* var, int ddof, cudaStream_t s);

}  // namespace uqlb
