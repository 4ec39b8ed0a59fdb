// Declarations shared by the storage-type translation units of the lattice-Boltzmann kernels
// (lbm_<type>.cu) and their dispatcher (lbm_launch.cu): the kernel parameter block and the table
// of launchers each storage type provides.  Internal; not part of the public ABI.
#pragma once

#include <cstdint>

#include "uqlb_internal.h"

namespace uqlb {

constexpr int kTileCols = 32;

struct KParams {
    void* arena;
    void* arena2;          // two-step scheme: second lattice
    int32_t* sel;          // two-step scheme: lattice holding each sample's state at the run's start
    const int32_t* row_base;  // row-strip kernel: first row of each sample in table order, [S + 1]
    const SampleDev* samples;
    const InitDev* init;
    const int32_t* steps_sorted;
    int32_t nsamples;
    int32_t uniform_tiles;
    const uint32_t* masks;
    float* side;
    double* side_d;
    double* bcpop;         // interpolated inlet/outlet: next state of the end columns
    double* partials;
    int32_t* counters;
    int32_t* done;
    int32_t* steps_run;
    double* cd_prev;
    int32_t* streak;
    const int64_t* step_counter;
    int32_t* n_done;
    unsigned int* bar_count;
    unsigned int* bar_gen;
    int32_t* bar_err;
    unsigned long long* tickets;
    int32_t test_withhold;
    int32_t dt;
    int32_t max_steps;
    int32_t stochastic;  // 16-bit storage: stochastic rounding of every population store
    int32_t spl;         // time steps per launch of the multi-step schemes (2 or 3)
    int32_t natural;     // the lattice holds the state in natural layout (cluster runs; finalize reads it so)
    // cluster runs: blocks per cluster, the widest sample's columns per block, the most rows
    int32_t cluster_size, cluster_cw, cluster_ny;
    // outputs
    void* fields;
    int64_t fields_ld;
    int32_t fields_dtype;
    double* qoi;
    double* series;
    double* series_cl;
    int64_t series_ld;
    int64_t qoi_every;
};

// Launchers of one population storage type (one translation unit per type, compiled in parallel).
// Resident blocks per SM of a row-strip kernel: the most that fit (registers, largest share), the
// default, the default shared-memory share per SM (KB) and the shared memory one block takes
// (bytes, with the 1 KB the system reserves per block).
struct StripBlocks {
    int max_b, def_b, def_kb, per_block;
};

struct StorageOps {
    cudaError_t (*init)(const KParams&, const BatchGeometry&, cudaStream_t);
    cudaError_t (*step)(const KParams&, const BatchGeometry&, bool odd, cudaStream_t);
    // two-step scheme: the row-strip kernel when g.strips is set, else the tile kernel
    cudaError_t (*two_step)(const KParams&, const BatchGeometry&, cudaStream_t, bool prepare_only);
    cudaError_t (*persistent)(const KParams&, const BatchGeometry&, int chunk, cudaStream_t);
    cudaError_t (*finalize)(const KParams&, const BatchGeometry&, cudaStream_t);
    cudaError_t (*inout)(const KParams&, const BatchGeometry&, cudaStream_t);
    cudaError_t (*bouzidi_force)(const KParams&, const BatchGeometry&, cudaStream_t);
    // cluster runs: the whole time loop of every sample in one launch (prepare_only: opt-ins only)
    cudaError_t (*cluster)(const KParams&, const BatchGeometry&, cudaStream_t, bool prepare_only);
    // three-step strips: blocks per SM at staging option `stage` (false: not a three-step strip batch)
    bool (*strip3_blocks)(const BatchGeometry&, int stage, StripBlocks*);
};
const StorageOps& storage_ops_f64();
const StorageOps& storage_ops_f32();
const StorageOps& storage_ops_f16();
const StorageOps& storage_ops_bf16();
const StorageOps& storage_ops_fx16();
// Blocks per cluster and columns per block of the last cluster launch (host side).
extern int g_cluster_choice[2];

// Streaming multiprocessors of the current device (queried once).
inline int sm_count() {
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 148;
    }
    return n;
}

}  // namespace uqlb
