/*
 * uqlb — ensemble lattice-Boltzmann uncertainty quantification on one GB300 (sm_103a).
 *
 * C ABI of libuqlb.so.  The calls follow the non-intrusive UQ workflow of
 * arXiv 2508.13867 (OpenLB-UQ), Sec. 7 and Algorithm 1: sample the uncertain inputs,
 * run the deterministic D2Q9 BGK solver for every sample, project the quantities of
 * interest onto the generalized polynomial chaos basis, report statistics.  The user
 * API of Sec. 8.1 (uniform/joint inputs, initializeMonteCarlo, initializeGPC,
 * getSamplingPoints, mean, std) maps onto uqlb_set_inputs, uqlb_init_mc,
 * uqlb_init_gpc, uqlb_get_samples, uqlb_mean_host and uqlb_std_host.
 *
 * Conventions shared by every call:
 *   - Every call returns a uqlb_status (0 = success); no C++ exception crosses the ABI.
 *     On failure uqlb_last_error() gives a one-line reason.
 *   - Ownership: the caller owns every pointer it passes.  Device buffers (suffix _dev)
 *     are plain device addresses, e.g. from torch tensors; host buffers are plain arrays.
 *     The library allocates no device memory for the run: the lattice arena, tables
 *     and reduction scratch live in a caller-supplied workspace whose size the
 *     *_workspace_bytes calls report.  The context owns only host memory and CUDA
 *     graph objects.
 *   - Streams: device work is enqueued asynchronously on the cudaStream_t passed as
 *     `stream` (NULL = legacy default stream).  Device-side errors (a sample that became
 *     unstable, a CUDA fault) surface at the next call that synchronises.
 *   - Layouts: all matrices are row-major.  Samples are indexed s = 0..S-1 in the order
 *     of uqlb_get_samples; gPC terms k = 0..K-1 in the order of uqlb_multi_indices.
 *   - Thread safety: a context must not be used from two host threads at once.
 */
#ifndef UQLB_H
#define UQLB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------------------------
 * Status codes and enums
 * ---------------------------------------------------------------------------------- */
typedef enum {
    UQLB_OK = 0,
    UQLB_ERR_ARG = -1,      /* invalid argument (null pointer, size out of range, ...) */
    UQLB_ERR_OOM = -2,      /* workspace too small or host allocation failed */
    UQLB_ERR_CUDA = -3,     /* a CUDA runtime call failed */
    UQLB_ERR_TIMEOUT = -4,  /* a bounded device wait gave up */
    UQLB_ERR_UNSTABLE = -5, /* a sample produced non-finite or non-positive density (or left the UQLB_FX16 range) */
    UQLB_ERR_STATE = -6     /* call out of order (e.g. project before init_gpc) */
} uqlb_status;

enum { UQLB_DIST_UNIFORM = 0 };               /* Sec. 6.1: uniform inputs (Legendre basis) */
enum { UQLB_BASIS_TOTAL = 0, UQLB_BASIS_TENSOR = 1 };
/* Sec. 6.3 quadrature rules: tensor-product Gauss-Legendre, or the Smolyak sparse grid over
 * nested Clenshaw-Curtis rules (pts_per_dim then gives the Smolyak level k; the grid integrates
 * total degree 2k + 1 exactly; 4 inputs at level 3 give the paper's 137 points). */
enum { UQLB_QUAD_GAUSS_LEGENDRE_TENSOR = 0, UQLB_QUAD_CLENSHAW_CURTIS_SMOLYAK = 1 };
enum { UQLB_METHOD_NONE = 0, UQLB_METHOD_MC = 1, UQLB_METHOD_GPC = 2 };
enum { UQLB_CASE_TGV = 0, UQLB_CASE_CHANNEL = 1, UQLB_CASE_TGV_PERTURBED = 2 };
/* Obstacle boundary scheme of the CHANNEL case (Sec. 8.1: the cylinder surface). */
enum { UQLB_OBSTACLE_HALFWAY = 0, UQLB_OBSTACLE_BOUZIDI = 1 };
/* Inlet/outlet scheme of the CHANNEL case (Sec. 8.1: interpolated velocity inlet and pressure
 * outlet). */
enum { UQLB_INOUT_FACE = 0, UQLB_INOUT_INTERPOLATED = 1 };
/* Parameters an uncertain input dimension may drive (uqlb_case.param_of_dim). */
enum {
    UQLB_PARAM_NU = 0,
    UQLB_PARAM_U0 = 1,
    UQLB_PARAM_ZETA2 = 2,
    UQLB_PARAM_ZETA3 = 3,
    UQLB_PARAM_PERT00 = 4, /* perturbed TGV amplitudes zeta_ij, relative to the sample's u0 */
    UQLB_PARAM_PERT01 = 5,
    UQLB_PARAM_PERT10 = 6,
    UQLB_PARAM_PERT11 = 7
};
/* Number formats: population storage, field outputs, projection inputs.  UQLB_FX16 is a population
 * storage format only: 16-bit fixed point, g_i = q d_c with q a signed 16-bit integer and one quantum
 * d_c per sample and velocity class c (rest, axis, diagonal), set from a bound on |g_i| over the run
 * (uqlb_fx16_quanta).  It spends all 15 magnitude bits on the range g actually takes, where FP16
 * keeps 11 significant bits and BF16 8, so its rounding error on the velocity field is several
 * times below FP16's and tens of times below BF16's at the same 2 bytes per population.  Stores
 * saturate at the ends of the range; a sample holding a saturated value at the end of its run gets
 * UQLB_ERR_UNSTABLE in its QoI status. */
enum { UQLB_F64 = 0, UQLB_F32 = 1, UQLB_F16 = 2, UQLB_BF16 = 3, UQLB_FX16 = 4 };
/* Rounding of 16-bit population stores.  Stochastic rounding (seeded by sample, node and step,
 * so runs reproduce) keeps the rounding error unbiased; nearest-even stagnates on fine lattices
 * where g changes by less than one unit in the last place per step.  FP32/FP64 ignore it. */
enum { UQLB_ROUND_AUTO = 0, UQLB_ROUND_NEAREST = 1, UQLB_ROUND_STOCHASTIC = 2 };
/* Columns of the per-sample scalar output qoi[S x UQLB_QOI_COLS] (FP64). */
enum {
    UQLB_QOI_K = 0,      /* normalised kinetic energy K(T) (Sec. 8.2, discrete form) */
    UQLB_QOI_MASS = 1,   /* sum of rho over fluid nodes at T */
    UQLB_QOI_MOMX = 2,   /* sum of rho u over fluid nodes at T */
    UQLB_QOI_MOMY = 3,   /* sum of rho v over fluid nodes at T */
    UQLB_QOI_CD = 4,     /* drag coefficient of the last step run (Sec. 8.1) */
    UQLB_QOI_CL = 5,     /* lift coefficient of the last step run */
    UQLB_QOI_STEPS = 6,  /* number of steps run */
    UQLB_QOI_STATUS = 7, /* 0 or UQLB_ERR_UNSTABLE */
    UQLB_QOI_COLS = 8
};

typedef struct uqlb_ctx uqlb_ctx;

/* One uncertain input (Sec. 6.1 Distribution): kind UQLB_DIST_UNIFORM on [a, b]. */
typedef struct {
    int32_t kind;
    int32_t reserved;
    double a, b;
} uqlb_dist;

/* One deterministic run (Sec. 7 "deterministic simulation"), all in lattice units.
 *   TGV (Sec. 8.2): periodic nx x ny lattice, u = u0 sin(kx)cos(ky) + amp2 (2k mode)
 *     + amp3 (3k mode), v the matching divergence-free field, k = 2 pi / n,
 *     rho = 1 + 3 p with p = u0^2/4 (cos 2kx + cos 2ky); K(t) normalised by u_ref.
 *   CHANNEL (Sec. 8.1): nx x ny nodes, halfway bounce-back walls at y = 0 and y = ny,
 *     parabolic velocity inlet of mean velocity u0 (peak 1.5 u0) at x = 0 with a
 *     1/2 (1 - cos(pi t / ramp_steps)) ramp, pressure outlet (rho = 1) at x = nx,
 *     staircase circular obstacle of centre (cyl_cx, cyl_cy) and radius cyl_r (node
 *     (x, y) solid iff its centre (x + 1/2, y + 1/2) lies strictly inside); C_D and
 *     C_L normalised by rho = 1, u0 and diameter 2 cyl_r.  With steady_tol > 0 a
 *     sample stops once |C_D(t) - C_D(t - qoi_every)| < steady_tol |C_D(t)| holds at
 *     steady_checks consecutive checks (FP32 resolves C_D to ~1e-7, so a tolerance below that
 *     needs several checks to avoid stopping on a chance coincidence).
 *     obstacle_bc selects the obstacle scheme: UQLB_OBSTACLE_HALFWAY (halfway bounce-back on
 *     the staircase, force 2 sum c_i f*_i) or UQLB_OBSTACLE_BOUZIDI, the linear interpolated
 *     bounce-back of Bouzidi, Firdaouss and Lallemand (2001) named by Sec. 8.1: a link from
 *     fluid node x along c_i meets the circle at the fraction q of its length and returns
 *     f_ibar(x, t+1) = 2q f*_i(x) + (1 - 2q) f_i(x, t+1) for q < 1/2 (f_i(x, t+1): the
 *     population streamed into x along c_i) or f*_i(x) / (2q) + (1 - 1/(2q)) f*_ibar(x) for
 *     q >= 1/2; the force is sum c_i (f*_i(x, t) + f_ibar(x, t+1)) after the stream.  Bouzidi
 *     samples run in UQLB_MODE_GRAPH only.
 *     inout_bc selects the inlet/outlet scheme: UQLB_INOUT_FACE (the moving-wall inlet and
 *     pressure outlet above, at the end faces) or UQLB_INOUT_INTERPOLATED, the finite-difference
 *     velocity-gradient conditions of Latt et al. (2008) cited by Sec. 8.1, on the end columns:
 *     after each stream every population of a node of column 0 (inlet) or nx - 1 (outlet) is
 *     replaced by f_i^eq(rho, u) - 3 w_i rho tau Q_i:S (Q_i = c_i c_i - I/3, S the strain rate
 *     by finite differences: second-order one-sided across the column, central along it,
 *     one-sided at its ends); inlet u = (parabola at the node centre, 0) with rho from the known
 *     populations by mass balance; outlet rho = 1, u_x from the known populations, u_y that of
 *     the node beside it.  Needs nx >= 6, ny >= 3 and the obstacle clear of the three end
 *     columns; UQLB_MODE_GRAPH only.
 *   TGV_PERTURBED (Sec. 8.3): periodic [0, 2 pi)^2 on nx x ny nodes x = 2 pi i / nx,
 *     u = -U cos 2x sin 2y, v = U sin 2x cos 2y, U = u0 + 1/4 sum_ij pert[2i+j] k_i(4x) k_j(4y)
 *     (k_0 = sin, k_1 = cos), p = -U^2/4 (cos 4x + cos 4y), rho = 1 + 3p; K(t) normalised by u_ref.
 * tau = 3 nu + 1/2 (Sec. 8.2), omega = 1 / tau. */
typedef struct {
    int32_t kind;        /* UQLB_CASE_TGV or UQLB_CASE_CHANNEL */
    int32_t nx, ny;      /* lattice size, 2 <= nx, ny <= 65536 */
    int32_t steady_checks; /* CHANNEL: consecutive checks that must pass (0 or 1: one check) */
    int64_t steps;       /* number of steps (TGV) or step cap (CHANNEL), 0 <= steps < 2^31 */
    double nu;           /* lattice viscosity, > 0 */
    double u0;           /* TGV amplitude or channel mean inflow velocity */
    double amp2, amp3;   /* TGV perturbation-mode amplitudes (absolute) */
    double u_ref;        /* TGV normaliser of K; 0 disables K */
    double cyl_cx, cyl_cy, cyl_r; /* CHANNEL obstacle; cyl_r <= 0: none */
    int64_t ramp_steps;  /* CHANNEL inflow ramp length (0: none) */
    double steady_tol;   /* CHANNEL steady-state tolerance (0: run to the cap) */
    double pert[4];      /* TGV_PERTURBED amplitudes zeta_00, zeta_01, zeta_10, zeta_11 (lattice units) */
    int32_t obstacle_bc; /* CHANNEL obstacle scheme, UQLB_OBSTACLE_HALFWAY or UQLB_OBSTACLE_BOUZIDI */
    int32_t inout_bc;    /* CHANNEL inlet/outlet scheme, UQLB_INOUT_FACE or UQLB_INOUT_INTERPOLATED */
} uqlb_sample;

/* Template of an ensemble: a uqlb_sample whose parameters are overridden per sample by
 * the uncertain inputs.  Input dimension d sets parameter param_of_dim[d]:
 *   UQLB_PARAM_NU -> nu;  UQLB_PARAM_U0 -> u0;
 *   UQLB_PARAM_ZETA2 / ZETA3 -> amp2 / amp3 = zeta * (the sample's u0);
 *   UQLB_PARAM_PERT00..11 -> pert[0..3] = zeta * (the sample's u0), i.e. zeta in units of u0 as in
 *   Sec. 8.3, where u0 = 1 and zeta ~ U(-0.025, 0.025). */
typedef struct {
    uqlb_sample base;
    int32_t param_of_dim[8];
} uqlb_case;

/* Options of a run.  Tile geometry: a tile is (32 x nodes_per_thread) columns by tile_rows rows
 * of one sample, run by 32 x tile_rows threads.  Compiled geometries, one-step scheme:
 * FP32/FP16/BF16 TGV-only batches tile_rows in {2, 4, 8} x nodes_per_thread in {1, 2, 4}; FP64
 * (8,1), (4,1), (4,2); batches with CHANNEL samples (8,1), (4,1).  Two-step scheme: FP32/FP16/
 * BF16 (4,4), (8,2), (8,4), (16,2), (16,4); FP64 (4,2), (8,1), (8,2).  Both 0: the geometry the
 * context's autotuner picked for this batch shape (uqlb_autotune), else the default. */
typedef struct {
    int32_t storage;          /* population storage: UQLB_F64, F32, F16, BF16 or FX16 (stored as f - w) */
    int32_t fields_dtype;     /* dtype of the field output M: UQLB_F64 or UQLB_F32 */
    int64_t qoi_every;        /* stride of the in-kernel QoI series (0: none) */
    int32_t chunk_steps;      /* steps per captured CUDA graph (even, 2..1024; 0: default 64) */
    int32_t tile_rows;        /* rows per tile (see above; 0: tuned or default) */
    int32_t nodes_per_thread; /* nodes per thread along x (see above; 0: tuned or default) */
    int32_t rounding;         /* 16-bit storage (F16, BF16, FX16): UQLB_ROUND_AUTO (= stochastic), NEAREST or STOCHASTIC */
    int64_t start_step;       /* 0: start from the initial field.  > 0: resume, i.e. continue the state
                                 a previous run left in the same workspace after start_step steps
                                 (same samples in the same order, options and workspace; each sample's
                                 `steps` is then its new total, which may order the samples differently
                                 by step count: a sample's state is kept by its position in the list).
                                 The workspace can be saved and restored between the two calls
                                 (checkpoint). */
    int32_t mode;             /* UQLB_MODE_GRAPH or UQLB_MODE_PERSISTENT (see below) */
    int32_t scheme;           /* time-stepping scheme, UQLB_SCHEME_* (see below) */
    /* Launch shape of the three-step row strips (ignored by the other kernels); each 0: the value
     * the context's autotuner picked for this batch shape, else the default. */
    int32_t strip_blocks_per_sm; /* resident blocks per SM (at most what fits; the grid is
                                    min(rows, blocks per SM x SMs) and each block takes an equal
                                    share of the rows) */
    int32_t strip_stage;      /* widths 64, 128, 256, 512, 1024: 1 = rows not staged, 2 = the next
                                 row staged in shared memory by cp.async, 3 = the next row loaded
                                 into registers (other widths: 0 only) */
    int32_t strip_smem_kb;    /* shared-memory share per SM in KB: 8, 16, 32, 64, 100, 132, 164, 196
                                 or 228 (the rest of the 256 KB is L1); raised to what the blocks
                                 per SM need */
} uqlb_run_opts;

/* Time-stepping scheme (the same BGK update of Sec. 3; they differ in how populations move
 * through memory).
 *   UQLB_SCHEME_ONE_STEP: one launch per time step, populations updated in place (AA order),
 *     72 B of HBM traffic per FP32 node update.  Every case kind and mode.
 *   UQLB_SCHEME_TWO_STEP: one launch per two time steps on two lattices (36 B of HBM traffic per
 *     FP32 node update).  Each node is collided at step t into shared memory, streamed from there,
 *     collided at step t + 1 and pushed to the other lattice.  Periodic (TGV, TGV_PERTURBED)
 *     batches in UQLB_MODE_GRAPH.  Two lattices: the workspace holds the second one, so a two- or
 *     three-step run needs twice the lattice memory of a one-step run (2.95 GB for 625 x 256^2 in
 *     FP32; uqlb_batch_workspace_bytes reports it).  FP32/FP64 results agree with the one-step
 *     scheme's to round-off (same formulas per node, a different operation order in the packed
 *     collisions), not bit for bit; 16-bit storage rounds half as often.  Two kernels:
 *       TWO_STEP_STRIPS: blocks walk full-width rows, keeping a ring of collided rows in shared
 *         memory (about 1 % of the nodes collided twice).  Every sample of the batch must have
 *         the same width nx, at most 2048 (1600 with FP32 storage, whose rows are also staged in
 *         shared memory; a block covers the row rounded up to 64 columns), with FP32, FP16, BF16 or
 *         FX16 storage; the tile geometry then serves only the initial state and the final fields.
 *       TWO_STEP_TILES: blocks take tiles of the tile geometry with a one-node halo (any size,
 *         FP64 too; the halo is collided twice, 27 % more collisions at tile 8 x 128).
 *     UQLB_SCHEME_TWO_STEP takes strips where the batch allows them, else tiles.
 *   UQLB_SCHEME_THREE_STEP_STRIPS: one launch per three time steps on the row strips, two rings of
 *     collided rows in shared memory (24 B of HBM traffic per FP32 node update); widths up to 1600
 *     (1280 with FP32 storage), the same storage formats and lattices as TWO_STEP_STRIPS.  A sample
 *     with fewer than three steps left runs two or one in its last launch.  With FP32 storage its
 *     fields equal the two-step strips' bit for bit (the same packed collisions of the same node
 *     pairs; FP32 rows pass through shared memory and HBM unrounded).
 *   UQLB_SCHEME_CLUSTER: CHANNEL samples with the halfway obstacle and the face inlet/outlet, FP32
 *     or 16-bit storage, UQLB_MODE_GRAPH: one thread-block cluster per sample holds the sample's
 *     lattice in shared memory (split into slabs of columns over up to 16 blocks, one copy, updated
 *     in place in AA order; slab edges through distributed shared memory) and runs its whole time
 *     loop, the steady-state test included, in one launch; HBM is touched to load the state and to
 *     write it back.  The largest sample's lattice, its link words and node lists must fit 16
 *     blocks' shared memory (about 220 KB per block: FP32 440 x 82 at 10 to 16 blocks, 16-bit up to
 *     about 860 x 160).  Cluster size: the one with the least estimated time over the clusters that
 *     run at once.  Fields equal the one-step scheme's bit for bit; C_D and C_L sum the same link
 *     forces in another order (FP32 round-off).  One workspace lattice, as ONE_STEP.
 *   UQLB_SCHEME_AUTO: the row strips for periodic FP32, FP16, BF16 and FX16 batches in graph mode,
 *     three steps per launch where the width allows it, else two, else TWO_STEP_TILES (measured on
 *     GB300, 625 x 256^2 ensemble, kernel GLUPS three-step strips / two-step strips / tiles /
 *     one-step: FP32 242 / 179 / 115 / 84, BF16 234 / 184 / 103 / 90, FP16 231 / 173 / 95 / 82,
 *     FX16 216 / 170 / - / -); CLUSTER for CHANNEL batches that allow it (FP32 9 x 440 x 82 cylinder
 *     samples: 60 against 24 GLUPS on ONE_STEP); ONE_STEP otherwise (FP64 is bound by the FP64
 *     rate).  In graph mode with FP32/FP16/BF16/FX16 storage a batch of unlike samples runs as
 *     groups of like samples, each on its own kernel and its own slice of the workspace
 *     (uqlb_batch_workspace_bytes counts them all).  The periodic groups run one after another on
 *     `stream`; the CHANNEL groups run at the same time on a second stream of the context (created at
 *     the first such run, highest priority), which `stream` waits for before any later work, so the
 *     latency-bound channel kernels share the SMs with the bandwidth-bound strips (uneven batch of
 *     256 TGV and 64 channel samples, BF16: 0.739 against 0.814 s one group after another).
 *     Groups: CHANNEL samples on CLUSTER where they fit (taken in order of size while the group's
 *     largest width and height fit), the other CHANNEL samples on ONE_STEP, periodic samples of each
 *     width the strips take on the strips, wider periodic samples on TWO_STEP_TILES.  Outputs keep the
 *     caller's rows.
 *     uqlb_last_run_geometry then reports UQLB_SCHEME_GROUPED.
 * A resumed run (start_step > 0) continues the state on any multi-step kernel (the strips and the
 * tiles, with two or three steps per launch, leave the same lattice layout); a one-step run resumes
 * on the one-step scheme only, a cluster run on the cluster scheme (it leaves the natural layout). */
enum {
    UQLB_SCHEME_AUTO = 0,
    UQLB_SCHEME_ONE_STEP = 1,
    UQLB_SCHEME_TWO_STEP = 2,
    UQLB_SCHEME_TWO_STEP_TILES = 3,
    UQLB_SCHEME_TWO_STEP_STRIPS = 4,
    UQLB_SCHEME_GROUPED = 5, /* reported only: the batch ran as groups (UQLB_SCHEME_AUTO) */
    UQLB_SCHEME_THREE_STEP_STRIPS = 6,
    UQLB_SCHEME_CLUSTER = 7
};

/* Execution of the time loop.
 *   UQLB_MODE_GRAPH: one launch per step, captured as CUDA graphs of chunk_steps launches.
 *   UQLB_MODE_PERSISTENT: one cooperative launch per chunk runs all its steps; tiles are handed
 *     out by a ticket counter (per-tile work queue) and steps are separated by a grid barrier
 *     whose wait is bounded (2 s): if it runs out, every sample's status becomes
 *     UQLB_ERR_TIMEOUT and uqlb_last_loop_time returns UQLB_ERR_TIMEOUT.
 *   UQLB_MODE_PERSISTENT_TEST_TIMEOUT: test hook of the bounded wait; block 0 never arrives at
 *     the barrier, so the run ends with UQLB_ERR_TIMEOUT after about 2 s. */
enum { UQLB_MODE_GRAPH = 0, UQLB_MODE_PERSISTENT = 1, UQLB_MODE_PERSISTENT_TEST_TIMEOUT = 2 };

/* ------------------------------------------------------------------------------------
 * Host building blocks (no device work)
 * ---------------------------------------------------------------------------------- */

/* n-point Gauss-Legendre rule on [-1, 1] (Sec. 6.3 Gauss quadrature): nodes x[n] ascending,
 * weights w[n] summing to 2.  1 <= n <= 64.  Newton iteration on the Legendre
 * three-term recurrence. */
int uqlb_gauss_legendre(int n, double* x, double* w);

/* Philox4x32-10 counter-based generator (Salmon et al., SC'11) used for the seeded Monte
 * Carlo draws of Sec. 8.1 (initializeMonteCarlo(N, dist, seed)).  out = bijection(ctr; key). */
int uqlb_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* Number of gPC terms K (Sec. 4.2 Eq. gPC) for `dim` inputs and polynomial `order`:
 * total degree (|alpha| <= order) or tensor (max alpha <= order). */
int uqlb_num_multi_indices(int dim, int order, int basis, int64_t* k);

/* Exponent set alpha[K x dim] ordered by |alpha|, then descending lexicographic order. */
int uqlb_multi_indices(int dim, int order, int basis, int32_t* alpha);

/* Lattice parameters of the Sec. 8.3 set-up (its table of simulation parameters): a domain of
 * length 2 pi resolved by n nodes, dx = 2 pi / (n - 1), dt = (Ma / sqrt 3) dx, physical nu = 1/Re,
 * tau = 3 nu dt / dx^2 + 1/2, lattice velocity of a unit physical velocity dt / dx.  n >= 2. */
int uqlb_unit_converter(int n, double ma, double re, double* dx, double* dt, double* tau,
                        double* u_lattice);

/* Quanta of the UQLB_FX16 storage for one sample, quanta[3] = (rest, axis, diagonal): margin x B_c / 32767
 * with B_c a bound on |g_i| of class c over the run, from the shifted D2Q9 equilibrium of Sec. 3 and its
 * first-order non-equilibrium part -3 tau w_i rho Q_i : grad u, given the sample's largest |c_i . u| = U,
 * velocity gradient G and density deviation R:  B_0 = 4/9 (R + (1 + R) 1.5 U^2),
 * B_axis = 1/9 (R + (1 + R)(3 U + 6 U^2 + 3 tau G)), B_diag = 1/36 (R + (1 + R)(3 U + 6 U^2 + 6 tau G)).
 * TGV: U = |u0| + |amp2| + |amp3|, G = k (|u0| + 2 |amp2| + 3 |amp3|) with k = 2 pi / min(nx, ny),
 * R = 1.5 U^2, margin 1.5; TGV_PERTURBED: U = |u0| + S / 4, G = k (2 |u0| + 1.5 S) with S = sum |pert|,
 * R = 1.5 U^2, margin 1.5 (with nx != ny the initial field is not divergence-free and its acoustic waves
 * need R = 2 sqrt(3) U); CHANNEL: U = 4 |u0|, G = U / 2, R = 6 |u0|, margin 1 (peak speeds, obstacle
 * shear and start-up pressure waves of the channel).  Each quantum is rounded to FP32 (the device keeps
 * it in FP32). */
int uqlb_fx16_quanta(const uqlb_sample* s, double* quanta);

/* Staircase obstacle mask of a CHANNEL sample, [ny x nx] bytes (1 = solid). */
int uqlb_obstacle_mask(const uqlb_sample* s, uint8_t* mask);

/* Eq. meanMCS on host data v[n]. */
int uqlb_mean_host(const double* v, int64_t n, double* out);

/* Square root of Eq. varMCS on host data: ddof = 1 gives 1/(n-1) (Eq. varMCS),
 * ddof = 0 gives Algorithm 1's 1/n. */
int uqlb_std_host(const double* v, int64_t n, int ddof, double* out);

/* ------------------------------------------------------------------------------------
 * UQ manager (Sec. 6.4 UncertaintyQuantification)
 * ---------------------------------------------------------------------------------- */

/* Create a context bound to CUDA device `cuda_device` (made current in every later call). */
int uqlb_create(uqlb_ctx** out, int cuda_device);
int uqlb_destroy(uqlb_ctx* ctx);

/* Reason of the last failure of `ctx` (or of a context-free call when ctx is NULL).
 * The string is owned by the library and valid until the next call on the same ctx. */
const char* uqlb_last_error(const uqlb_ctx* ctx);

/* Joint distribution of `dim` independent inputs (1 <= dim <= 8), Sec. 8.3 `joint`. */
int uqlb_set_inputs(uqlb_ctx* ctx, int dim, const uqlb_dist* d);

/* Monte Carlo sample set (Sec. 4.1): n seeded draws, counter (s lo, s hi, dim, 0),
 * key = seed, u = ((x1 << 32 | x0) >> 11) 2^-53, z = a + (b - a) u.  Weights 1/n. */
int uqlb_init_mc(uqlb_ctx* ctx, int64_t n, uint64_t seed);

/* Quasi Monte Carlo sample set (Sec. 4.1): n Halton points (radical inverses of s + skip in the
 * first `dim` primes), z = a + (b - a) u, weights 1/n; statistics use the Monte Carlo estimators.
 * 1 <= n <= 2^24, skip >= 0. */
int uqlb_init_qmc(uqlb_ctx* ctx, int64_t n, int64_t skip);

/* Stochastic collocation (Sec. 4.2, Sec. 8.1 initializeGPC(order, N, dist)): tensor
 * Gauss-Legendre grid with pts_per_dim nodes per input (last input fastest), weights of
 * the uniform probability measure, orthonormal Legendre chaos of `order` (`basis`
 * total or tensor).  Builds W[k, s] = a_s Phi_k(xi_s) (Eq. coef_discrete).  With quad =
 * UQLB_QUAD_CLENSHAW_CURTIS_SMOLYAK the nodes are the Smolyak grid of level pts_per_dim (0..6),
 * ordered lexicographically by their indices on the finest one-dimensional grid; sparse-grid
 * weights can be negative. */
int uqlb_init_gpc(uqlb_ctx* ctx, int order, int pts_per_dim, int basis, int quad);

int uqlb_num_samples(const uqlb_ctx* ctx, int64_t* n);
int uqlb_num_terms(const uqlb_ctx* ctx, int* k);

/* Sampling points (Sec. 8.1 getSamplingPoints): z[S x dim] physical values, xi[S x dim]
 * reference values in [-1, 1], a[S] quadrature weights (1/S for MC).  Any output may be NULL. */
int uqlb_get_samples(const uqlb_ctx* ctx, double* z, double* xi, double* a);

/* Host copy of the projection matrix W[K x S] (gPC only). */
int uqlb_get_weight_matrix(const uqlb_ctx* ctx, double* w);

/* ------------------------------------------------------------------------------------
 * Deterministic solves over the ensemble (Sec. 7, Algorithm 1 loop)
 * ---------------------------------------------------------------------------------- */

/* Workspace needed by uqlb_run_batch for these samples and options (with both geometry fields
 * 0: enough for every compiled geometry, so that tuned runs fit). */
int uqlb_batch_workspace_bytes(const uqlb_sample* samples, int64_t n, const uqlb_run_opts* opts,
                               size_t* bytes);

/* Run n independent samples on the device: initialise every lattice at equilibrium, step all
 * samples with the collision, streaming, boundaries and QoI reductions fused into the step kernels
 * of the run's scheme (uqlb_run_opts.scheme: in place in AA order with one launch per step, or two
 * lattices with two or three steps per launch; under UQLB_SCHEME_AUTO periodic FP32/16-bit batches
 * take two lattices, so size the workspace with uqlb_batch_workspace_bytes for the same options),
 * and write the results.
 *   workspace_dev / workspace_bytes: scratch of at least uqlb_batch_workspace_bytes bytes,
 *     256-byte aligned; contents on entry are ignored.
 *   fields_dev: optional (NULL to skip), row s = [u (ny*nx), v (ny*nx), K(T)] of sample s in
 *     fields_dtype with row stride fields_ld >= 2 nx ny + 1 elements; requires all samples to
 *     share nx, ny.  Obstacle nodes hold 0.
 *   qoi_dev: optional FP64 [n x UQLB_QOI_COLS] per-sample scalars.
 *   series_dev: optional FP64 [n x series_ld]; TGV: K(j qoi_every) in column j (j = 0 is t = 0);
 *     CHANNEL: C_D after step j qoi_every in column j - 1.  Unwritten entries are untouched.
 *   series_cl_dev: optional FP64 [n x series_ld], CHANNEL lift at the same times.
 * Returns after enqueueing; for CHANNEL samples with steady_tol > 0 it synchronises `stream`
 * between graph launches to test for convergence. */
int uqlb_run_batch(uqlb_ctx* ctx, const uqlb_sample* samples, int64_t n, const uqlb_run_opts* opts,
                   void* workspace_dev, size_t workspace_bytes, void* fields_dev, int64_t fields_ld,
                   double* qoi_dev, double* series_dev, double* series_cl_dev, int64_t series_ld,
                   void* stream);

/* Launch-shape autotuner.  For this batch shape, time `trial_steps` (>= 2, even) steps of every
 * candidate launch shape on the device (after an equilibrium initialisation and one untimed
 * launch, CUDA events on `stream`, best of three passes) and keep the fastest in the context;
 * later runs of a batch with the same storage, kinds, sample count and node count use it for the
 * fields they pass as 0.
 * Candidates: on the tile kernels every compiled tile geometry; on the three-step row strips (the
 * default for periodic batches of one width) the staging option x resident blocks per SM (the
 * most that fit and up to three fewer) x shared-memory share (the smallest holding the blocks,
 * and the largest), the tile geometry staying at its default.  Outputs (any may be NULL): the
 * chosen tile_rows / nodes_per_thread, and for each candidate c < *n_tried: rows_tried[c],
 * npt_tried[c], ms_per_step[c] (arrays of capacity 16; the full list, strip knobs included, from
 * uqlb_autotune_report).  The workspace must hold uqlb_batch_workspace_bytes for opts with the
 * geometry fields 0; its contents are overwritten.  Synchronises `stream`.  A batch that runs as
 * groups is tuned group by group; the outputs describe the group with the most node updates. */
int uqlb_autotune(uqlb_ctx* ctx, const uqlb_sample* samples, int64_t n, const uqlb_run_opts* opts,
                  void* workspace_dev, size_t workspace_bytes, int trial_steps, int32_t* tile_rows,
                  int32_t* nodes_per_thread, int32_t* rows_tried, int32_t* npt_tried,
                  double* ms_per_step, int32_t* n_tried, void* stream);

/* One candidate of the last uqlb_autotune call (of its largest group). */
typedef struct {
    int32_t scheme;           /* UQLB_SCHEME_* of the kernel the candidate ran */
    int32_t tile_rows, nodes_per_thread;
    int32_t strip_blocks_per_sm, strip_stage, strip_smem_kb;  /* 0 off the three-step strips */
    double ms_per_step;       /* best of three passes */
} uqlb_tune_candidate;

/* The candidates of the context's last uqlb_autotune call (host): up to `cap` into `out` (may be
 * NULL when cap is 0), their count into *n and the index of the chosen one into *chosen (-1: no
 * autotune yet). */
int uqlb_autotune_report(const uqlb_ctx* ctx, uqlb_tune_candidate* out, int32_t cap, int32_t* n,
                         int32_t* chosen);

/* Build the per-sample runs of the context's sample set from a case template (host). */
int uqlb_ensemble_samples(const uqlb_ctx* ctx, const uqlb_case* c, uqlb_sample* out);

/* Workspace for uqlb_run_ensemble (the batch workspace of the ensemble's samples). */
int uqlb_ensemble_workspace_bytes(const uqlb_ctx* ctx, const uqlb_case* c, const uqlb_run_opts* opts,
                                  size_t* bytes);

/* uqlb_ensemble_samples followed by uqlb_run_batch over all S samples. */
int uqlb_run_ensemble(uqlb_ctx* ctx, const uqlb_case* c, const uqlb_run_opts* opts,
                      void* workspace_dev, size_t workspace_bytes, void* fields_dev,
                      int64_t fields_ld, double* qoi_dev, double* series_dev,
                      double* series_cl_dev, int64_t series_ld, void* stream);

/* Plain per-sample FP64 path: one sample at a time, one kernel launch per step on two
 * lattices (pull streaming), QoIs in separate kernels.  Same outputs as uqlb_run_batch with
 * storage UQLB_F64 (fields in FP64).  Serves as the unbatched, unfused FP64 comparator. */
int uqlb_plain_workspace_bytes(const uqlb_sample* samples, int64_t n, size_t* bytes);
int uqlb_run_plain_f64(uqlb_ctx* ctx, const uqlb_sample* samples, int64_t n, int64_t qoi_every,
                       void* workspace_dev, size_t workspace_bytes, double* fields_dev,
                       int64_t fields_ld, double* qoi_dev, double* series_dev, int64_t series_ld,
                       void* stream);

/* Device time of the time loop of the last uqlb_run_batch / uqlb_run_ensemble on this context
 * (returns UQLB_ERR_TIMEOUT if a bounded wait of a persistent run gave up),
 * measured with CUDA events recorded on the caller's stream around the graph launches of the
 * loop (so it covers the fused step kernels and nothing else of the run).  steps: time steps of
 * the loop; launches: kernels the whole run enqueued (init, steps, counter advances, finalize).
 * Synchronises on the end event.  Any output may be NULL. */
int uqlb_last_loop_time(uqlb_ctx* ctx, double* ms, int64_t* steps, int64_t* launches);

/* Scheme the last uqlb_run_batch / uqlb_run_ensemble on this context ran (UQLB_SCHEME_ONE_STEP,
 * UQLB_SCHEME_TWO_STEP_TILES, UQLB_SCHEME_TWO_STEP_STRIPS, UQLB_SCHEME_THREE_STEP_STRIPS,
 * UQLB_SCHEME_CLUSTER, or UQLB_SCHEME_GROUPED for a batch run as groups) and its tile geometry (of the
 * first group; for UQLB_SCHEME_CLUSTER the blocks per cluster and the columns per block).  Any output
 * may be NULL; UQLB_ERR_STATE before the first run. */
int uqlb_last_run_geometry(const uqlb_ctx* ctx, int32_t* scheme, int32_t* tile_rows, int32_t* nodes_per_thread);

/* ------------------------------------------------------------------------------------
 * Statistical-solution distance (Sec. 8.3)
 * ---------------------------------------------------------------------------------- */

/* 1-Wasserstein distance between the empirical distributions of the speed |u| = sqrt(u^2 + v^2)
 * over all samples and nodes of two field sets, e.g. two resolutions of one ensemble (Sec. 8.3:
 * W1 of the numerical statistical solutions of |u|).  Set X is M_X[s_X x ld_X] in dtype_X (F64 or
 * F32) with rows [u (nodes_X values), v (nodes_X values), ...] as uqlb_run_batch writes them.
 * Both sets are binned into `bins` (1..2^24) equal bins over [0, largest speed of both]; the
 * distance is the integral of |F_a - F_b| over those bins.  Binning moves each value by less
 * than one bin, so the result is within one bin width (written to bound_host) of the exact
 * distance.  Non-finite speeds (samples that became unstable) are left out and counted in
 * nonfinite_host[0] / [1] (may be NULL); a set with no finite speed gives NaN.  Writes the
 * distance to out_host; synchronises `stream`. */
int uqlb_w1_workspace_bytes(int bins, size_t* bytes);
int uqlb_w1_speed(uqlb_ctx* ctx, const void* a_dev, int dtype_a, int64_t s_a, int64_t nodes_a, int64_t ld_a,
                  const void* b_dev, int dtype_b, int64_t s_b, int64_t nodes_b, int64_t ld_b, int bins,
                  void* workspace_dev, size_t workspace_bytes, double* out_host, double* bound_host,
                  int64_t* nonfinite_host, void* stream);

/* ------------------------------------------------------------------------------------
 * Postprocessing (Sec. 4, Algorithm 1 statistics)
 * ---------------------------------------------------------------------------------- */

/* Device workspace of uqlb_project / uqlb_stats for the dense contraction (holds W on the device). */
int uqlb_post_workspace_bytes(const uqlb_ctx* ctx, size_t* bytes);

/* Device workspace with which uqlb_project takes its fastest contraction for n_fields fields: on a
 * tensor Gauss-Legendre sample set with at most 16 points per input and degree at most 8, the tables
 * and the intermediate buffers of the sum-factorized contraction (for the 4-D total-degree-4 basis on
 * 5^4 points, 1000 rows of n_fields FP64 values); otherwise uqlb_post_workspace_bytes.  Requires
 * uqlb_init_gpc. */
int uqlb_project_workspace_bytes(const uqlb_ctx* ctx, int64_t n_fields, size_t* bytes);

/* gPC coefficients (Eq. coef_discrete, gamma_k = 1): coeffs[k, f] = sum_s W[k, s] M[s, f],
 * accumulated in FP64.  m_dev: [S x n_fields] in `dtype` (UQLB_F64 or UQLB_F32) with row
 * stride m_ld; coeffs_dev: FP64 [K x n_fields] dense.  Requires uqlb_init_gpc.
 * Two contractions, equal to FP64 round-off:
 *   sum-factorized, on a tensor Gauss-Legendre sample set (at most 16 points per input, degree at
 *     most 8) when the
 *     workspace holds uqlb_project_workspace_bytes for n_fields (8-byte aligned).  W[k, s] is then
 *     the product over the inputs of G[alpha_kq][s_q] = (w_s / 2) phi_a(x_s), so the sum over the
 *     samples is taken one input at a time, the last input first: for d = 4, order 4, 5 points,
 *     6 225 instead of 43 750 FP64 multiply-adds per field (d launches);
 *   dense, [K x S] x [S x n_fields], with a workspace below that (uqlb_post_workspace_bytes suffices)
 *     and for every other sample set; on one input the two coincide up to the order of operations.
 * uqlb_last_projection reports which one the last call took. */
int uqlb_project(uqlb_ctx* ctx, const void* m_dev, int dtype, int64_t n_fields, int64_t m_ld,
                 double* coeffs_dev, void* workspace_dev, size_t workspace_bytes, void* stream);

/* The contraction of the last uqlb_project on ctx: 0 dense, 1 sum-factorized. */
int uqlb_last_projection(const uqlb_ctx* ctx, int32_t* kind);

/* uqlb_project for callers that cannot allocate device memory.  The paper has no counterpart:
 * this is an interface for hosts such as code running under a fixed device-memory budget,
 * threads that must not enter an allocator, or embeddings that only hand over their own input
 * and output buffers.  Same arguments and result as uqlb_project, but no workspace: the weight
 * matrix W is staged in a fixed device array inside the library (1 MiB, K x S <= 131072
 * weights; larger sample sets return UQLB_ERR_ARG and need uqlb_project).  No device memory is
 * allocated or freed.  The array exists once per GPU that loads the library and stays until
 * the process exits.  The weights are copied from the context's host memory (pageable) on the
 * stream, so neither this call nor uqlb_project can be captured into a CUDA graph.  The first call
 * on a device looks up the array's device address.  The library keeps that address for the life of the
 * process: it must not outlive a reset of the device (cudaDeviceReset), which would leave the kept
 * address pointing at memory that no longer holds the array.  All calls share the one array: calls that
 * overlap on the GPU (e.g. on two streams) race and must be ordered by the caller.  Each call
 * overwrites every weight it reads, so no contents carry over between calls. */
int uqlb_project_noalloc(uqlb_ctx* ctx, const void* m_dev, int dtype, int64_t n_fields, int64_t m_ld,
                         double* coeffs_dev, void* stream);

/* Sample-level parallelism across GPUs (the paper's Sec. 9 hybrid parallelism runs samples
 * independently; the statistics are its only exchange).  A sharded run gives each GPU a contiguous
 * block of samples s0 .. s0 + count - 1 of the context's sample set (uqlb_ensemble_samples lists
 * them; uqlb_run_batch runs the block, whose rows are then 0 .. count - 1), and:
 *   gPC: uqlb_project_block forms the block's partial coefficients
 *     partial[k, f] = sum_{s < count} W[k, s0 + s] M[s, f] (Eq. coef_discrete restricted to the
 *     block, FP64); the coefficients are linear in the samples, so the sum of the partials of blocks
 *     that cover 0 .. S - 1 (one all-reduce) equals uqlb_project's, and uqlb_stats then gives the
 *     mean and variance.  m_dev: [count x n_fields] (row stride m_ld) in dtype F64 or F32;
 *     coeffs_dev: FP64 [K x n_fields]; the workspace is uqlb_post_workspace_bytes.  Synchronises
 *     `stream` after the weight upload.  UQLB_ERR_ARG for a block outside 0 .. S - 1.
 *   MC: uqlb_block_moments gives the block's mean[f] (Eq. meanMCS over its n_rows rows) and
 *     m2[f] = sum over the rows of (M[s, f] - mean[f])^2 (two passes, FP64); blocks merge exactly by the
 *     pairwise update of Chan, Golub and LeVeque (n = n_a + n_b, delta = mean_b - mean_a,
 *     mean = mean_a + delta n_b / n, m2 = m2_a + m2_b + delta^2 n_a n_b / n), and Eq. varMCS is
 *     m2 / (N - ddof).  The call needs no sample set (any context serves).
 * uqlb_get_weight_block copies the block's columns of W to the host, [K x count], as
 * uqlb_project_block uploads them. */
int uqlb_get_weight_block(const uqlb_ctx* ctx, int64_t s0, int64_t count, double* w);
int uqlb_project_block(uqlb_ctx* ctx, const void* m_dev, int dtype, int64_t n_fields, int64_t m_ld, int64_t s0,
                       int64_t count, double* coeffs_dev, void* workspace_dev, size_t workspace_bytes, void* stream);
int uqlb_block_moments(uqlb_ctx* ctx, const void* m_dev, int dtype, int64_t n_rows, int64_t n_fields, int64_t m_ld,
                       double* mean_dev, double* m2_dev, void* stream);

/* Statistics per field, FP64 outputs mean_dev[n_fields], var_dev[n_fields].
 *   gPC context: input is coeffs_dev [K x n_fields] FP64; mean = c_0 (Eq. gpc_mean),
 *     var = sum_{k >= 1} c_k^2 (Eq. gpc_std squared); dtype must be UQLB_F64, ddof ignored.
 *   MC context: input is M [S x n_fields] (ld = m_ld) in `dtype`; mean by Eq. meanMCS,
 *     var by Eq. varMCS with divisor S - ddof (two passes, FP64). */
int uqlb_stats(uqlb_ctx* ctx, const void* in_dev, int dtype, int64_t n_fields, int64_t m_ld,
               double* mean_dev, double* var_dev, int ddof, void* stream);

/* End-to-end UQ through host buffers (Algorithm 1 as one call): runs the ensemble of the
 * context's samples, projects (gPC) or averages (MC) the fields [u, v, K] and copies
 * mean_host / var_host [2 nx ny + 1] (and, for gPC and when not NULL, coeffs_host
 * [K x (2 nx ny + 1)]) back to the host.  Device scratch comes from workspace_dev
 * (uqlb_uq_workspace_bytes); synchronises `stream` before returning. */
int uqlb_uq_workspace_bytes(const uqlb_ctx* ctx, const uqlb_case* c, const uqlb_run_opts* opts,
                            size_t* bytes);
int uqlb_run_uq_host(uqlb_ctx* ctx, const uqlb_case* c, const uqlb_run_opts* opts,
                     void* workspace_dev, size_t workspace_bytes, double* mean_host,
                     double* var_host, double* coeffs_host, double* qoi_host, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* UQLB_H */
