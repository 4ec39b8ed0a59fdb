// Dispatch of the lattice-Boltzmann launchers by population storage type, the kernel parameter
// block, and the small kernels that do not depend on the storage type (arXiv 2508.13867, Sec. 7
// time loop).  The step, init and finalize kernels live in one translation unit per storage
// type (lbm_<type>.cu).
#include <algorithm>

#include "lbm_kernels.cuh"

namespace uqlb {

int g_cluster_choice[2] = {0, 0};

void last_cluster_choice(int* blocks, int* cols) {
    *blocks = g_cluster_choice[0];
    *cols = g_cluster_choice[1];
}

namespace {

// After the finalize of a two-step run: the lattice that now holds each sample's state (both
// arrays are indexed by the sample's slot).
__global__ void commit_kernel(KParams p) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < p.nsamples; k += gridDim.x * blockDim.x)
        p.sel[k] ^= launches_of(p.steps_run[k], (int)p.step_counter[1], p.spl) & 1;
}

__global__ void advance_kernel(int64_t* counter, int chunk) { *counter += chunk; }

// Resuming a run: samples that have not stopped take their new step totals.
__global__ void resume_kernel(KParams p) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < p.nsamples; j += gridDim.x * blockDim.x)
        if (!p.done[p.samples[j].slot]) p.steps_run[p.samples[j].slot] = p.samples[j].steps;
}

const StorageOps& ops_of(int storage) {
    switch (storage) {
        case UQLB_F64: return storage_ops_f64();
        case UQLB_F32: return storage_ops_f32();
        case UQLB_F16: return storage_ops_f16();
        case UQLB_FX16: return storage_ops_fx16();
        default: return storage_ops_bf16();
    }
}

KParams make_params(const BatchBuffers& b, const BatchGeometry& g, const RunOutputs* o, int dt) {
    KParams p{};
    p.arena = b.arena;
    p.arena2 = b.arena2;
    p.sel = b.sel;
    p.row_base = b.row_base;
    p.samples = b.samples;
    p.init = b.init;
    p.steps_sorted = b.steps_sorted;
    p.nsamples = (int32_t)g.nsamples;
    p.uniform_tiles = g.uniform_tiles;
    p.masks = b.masks;
    p.side = b.side;
    p.side_d = b.side_d;
    p.bcpop = b.bcpop;
    p.partials = b.partials;
    p.counters = b.counters;
    p.done = b.done;
    p.steps_run = b.steps_run;
    p.cd_prev = b.cd_prev;
    p.streak = b.streak;
    p.step_counter = b.step_counter;
    p.n_done = b.active_flag;
    p.bar_count = b.bar_count;
    p.bar_gen = b.bar_gen;
    p.bar_err = b.bar_err;
    p.tickets = b.tickets;
    p.test_withhold = g.test_withhold;
    p.dt = dt;
    p.max_steps = g.max_steps;
    p.stochastic = g.stochastic;
    p.spl = g.spl > 0 ? g.spl : 2;
    p.natural = g.cluster;
    if (o != nullptr) {
        p.fields = o->fields;
        p.fields_ld = o->fields_ld;
        p.fields_dtype = o->fields_dtype;
        p.qoi = o->qoi;
        p.series = o->series;
        p.series_cl = o->series_cl;
        p.series_ld = o->series_ld;
        p.qoi_every = o->qoi_every;
    }
    return p;
}

}  // namespace

bool strip_supported(int storage, int nx) {
    if (storage == UQLB_F64 || nx < 2) return false;
    const int rw = 2 * strip_threads(nx);  // the ring's width: nx rounded up to 64 columns
    return rw <= (storage == UQLB_F32 ? StripTune<float>::max_nx : StripTune<__half>::max_nx);
}

bool strip3_supported(int storage, int nx) {
    if (storage == UQLB_F64 || nx < 2) return false;
    const int rw = 2 * strip_threads(nx);
    return rw <= (storage == UQLB_F32 ? Strip3Tune<float>::max_nx : Strip3Tune<__half>::max_nx);
}

bool cluster_fits(int storage, int nx, int ny) {
    if (storage == UQLB_F64 || nx < 1 || ny < 1) return false;
    const size_t eb = storage == UQLB_F32 ? 4 : 2;
    for (int c = 1; c <= 16; ++c) {
        const int cw = (nx + c - 1) / c;  // rows of exactly cw columns where no padded width fits
        const size_t smem = (9 * (size_t)cw * ny * eb + 15) / 16 * 16 + 2 * (size_t)cw * ny * sizeof(uint32_t);
        if (smem <= 227 * 1024 - 4096) return true;
    }
    return false;
}

bool strip3_blocks(const BatchGeometry& g, int stage, int* max_b, int* def_b, int* def_kb, int* per_block) {
    StripBlocks b{};
    if (!ops_of(g.storage).strip3_blocks(g, stage, &b)) return false;
    *max_b = b.max_b;
    *def_b = b.def_b;
    *def_kb = b.def_kb;
    *per_block = b.per_block;
    return true;
}

bool geometry_supported2(int storage, int tile_rows, int npt) {
    const int tr = tile_rows, n = npt;
    if (storage == UQLB_F64) return (tr == 4 && n == 2) || (tr == 8 && (n == 1 || n == 2));
    return (tr == 4 && n == 4) || ((tr == 8 || tr == 16) && (n == 2 || n == 4));
}

bool geometry_supported(int storage, bool mixed, int tile_rows, int npt) {
    const int tr = tile_rows, n = npt;
    if (mixed) return n == 1 && (tr == 8 || tr == 4);
    if (storage == UQLB_F64) return (n == 1 && (tr == 8 || tr == 4)) || (n == 2 && tr == 4);
    return (tr == 2 || tr == 4 || tr == 8) && (n == 1 || n == 2 || n == 4);
}

cudaError_t prepare_step2(const BatchGeometry& g) {
    KParams p{};
    return ops_of(g.storage).two_step(p, g, nullptr, true);
}

cudaError_t launch_step2(const BatchBuffers& b, const BatchGeometry& g, const RunOutputs& o, int dt, cudaStream_t s) {
    return ops_of(g.storage).two_step(make_params(b, g, &o, dt), g, s, false);
}

cudaError_t launch_commit(const BatchBuffers& b, const BatchGeometry& g, cudaStream_t s) {
    KParams p = make_params(b, g, nullptr, 0);
    const int grid = (int)std::min<int64_t>((g.nsamples + 255) / 256, 1024);
    commit_kernel<<<grid, 256, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_init(const BatchBuffers& b, const BatchGeometry& g, cudaStream_t s) {
    return ops_of(g.storage).init(make_params(b, g, nullptr, 0), g, s);
}

cudaError_t launch_inout(const BatchBuffers& b, const BatchGeometry& g, int dt, cudaStream_t s) {
    return ops_of(g.storage).inout(make_params(b, g, nullptr, dt), g, s);
}

cudaError_t launch_bouzidi_force(const BatchBuffers& b, const BatchGeometry& g, const RunOutputs& o, int dt,
                                 int base_parity, cudaStream_t s) {
    (void)base_parity;  // the kernel takes the AA layout from the parity of the step index
    return ops_of(g.storage).bouzidi_force(make_params(b, g, &o, dt), g, s);
}

cudaError_t launch_step(const BatchBuffers& b, const BatchGeometry& g, const RunOutputs& o, int dt, int base_parity,
                        cudaStream_t s) {
    const bool odd = ((dt + base_parity) & 1) != 0;
    return ops_of(g.storage).step(make_params(b, g, &o, dt), g, odd, s);
}

cudaError_t launch_persistent(const BatchBuffers& b, const BatchGeometry& g, const RunOutputs& o, int chunk,
                              cudaStream_t s) {
    return ops_of(g.storage).persistent(make_params(b, g, &o, 0), g, chunk, s);
}

cudaError_t launch_resume(const BatchBuffers& b, const BatchGeometry& g, cudaStream_t s) {
    KParams p = make_params(b, g, nullptr, 0);
    resume_kernel<<<(int)std::min<int64_t>((g.nsamples + 255) / 256, 1024), 256, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_advance(const BatchBuffers& b, int chunk, cudaStream_t s) {
    advance_kernel<<<1, 1, 0, s>>>(b.step_counter, chunk);
    return cudaGetLastError();
}

cudaError_t launch_cluster(const BatchBuffers& b, const BatchGeometry& g, const RunOutputs& o, cudaStream_t s) {
    return ops_of(g.storage).cluster(make_params(b, g, &o, 0), g, s, false);
}

cudaError_t launch_finalize(const BatchBuffers& b, const BatchGeometry& g, const RunOutputs& o,
                            cudaStream_t s) {
    return ops_of(g.storage).finalize(make_params(b, g, &o, 0), g, s);
}

}  // namespace uqlb
