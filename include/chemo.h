/*
 * chemo.h -- C ABI of the GB300 (sm_103a) particle step of the hybrid
 * chemotaxis model of Bruna, Maini & Robinson, "Particle-based simulations of
 * reaction-diffusion processes with Aboria" (arXiv:1805.11007).
 *
 * One simulation object holds N cells (point particles of up to 8 species)
 * in a 2D or 3D box and, optionally, the chemical concentration c on a
 * regular grid. One step (chemo_step) advances both by dt:
 *
 *   a1  bin each cell into a cell list (Sect. 2.2, 3.1: neighbourhood search)
 *   a2  counting-sort the cells by bin (row-major) and build the bin offsets
 *   a3  sum the finite-range soft repulsion over neighbouring bins
 *       (Sect. 3.2 interaction loop; pair term of Eq. (1a)/(1b))
 *   a4  interpolate the central-difference gradient of c^n to each cell
 *       (Sect. 2.3, 3.5 D1x/D1y, 3.6) for the chemotactic drift of Eq. (1b)
 *   a5  Euler-Maruyama move (Eq. (2)) with reflecting walls (Sect. 3.2) or a
 *       periodic box with unwrapped displacement (Sect. 4)
 *   a6  deposit the secretion (and consumption) of the moved cells on the
 *       grid by cloud-in-cell weights (Sect. 2.3, random measures Eq. (1e))
 *   a7  explicit PDE step of Eq. (1d): centred differences in space, forward
 *       Euler in time (Sect. 3.5), with substeps when stability requires.
 *
 * Conventions (every function):
 *   - returns an int status (CHEMO_OK = 0, negative on error) and never
 *     throws; chemo_last_error() gives a thread-local message;
 *   - pointers passed in are borrowed for the duration of the call only;
 *     the library owns all device memory of a simulation;
 *   - `mem_kind` says where a caller buffer lives: CHEMO_MEM_HOST (pageable
 *     or pinned host memory; the call synchronises the stream before it
 *     returns) or CHEMO_MEM_DEVICE (device memory of the current device; the
 *     call is asynchronous on `stream`);
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream); work is
 *     ordered on it. Errors found on the device (non-finite position, bin or
 *     buffer overflow, a bounded wait that ran out) are latched in the
 *     simulation and reported by the next chemo_check / chemo_read_* call.
 *   - Particle arrays are indexed by particle id (0..n-1, the order given to
 *     chemo_create); positions are n x dim row-major float32; grids are
 *     C-order [z][y][x] float32 with x fastest (2D: [y][x]).
 */
#ifndef CHEMO_H
#define CHEMO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CHEMO_ABI_VERSION 1
#define CHEMO_MAX_SPECIES 8

/* Status codes. */
enum {
    CHEMO_OK = 0,
    CHEMO_EINVAL = -1,     /* invalid argument or parameter set */
    CHEMO_ENOMEM = -2,     /* device or host allocation failed */
    CHEMO_ECUDA = -3,      /* a CUDA runtime call failed */
    CHEMO_EDOMAIN = -4,    /* a particle left the domain */
    CHEMO_ENONFINITE = -5, /* a non-finite position appeared */
    CHEMO_EOVERFLOW = -6,  /* a bin, buffer or index range overflowed */
    CHEMO_ETIMEOUT = -7,   /* a bounded device-side wait gave up */
    CHEMO_ENOTSUP = -8     /* option not supported by this build */
};

enum { CHEMO_MEM_HOST = 0, CHEMO_MEM_DEVICE = 1 };

/* Model parameters, copied at chemo_create / chemo_set_params.
 * Defaults: zero-fill the struct, then set struct_size = sizeof(chemo_params)
 * and the fields below. Per-species arrays use entries [0, n_species). */
typedef struct chemo_params {
    uint32_t struct_size;        /* sizeof(chemo_params), for ABI checks */
    int32_t dim;                 /* 2 or 3 (the paper's model is 2D, Sect. 2) */
    int32_t boundary;            /* 0 reflecting walls (Sect. 3.2), 1 periodic (Sect. 4) */
    double lo[3], hi[3];         /* domain box [lo, hi] per axis */
    int32_t n_species;           /* 1..8 (the paper: alpha = 0, beta = 1) */
    float diameter[CHEMO_MAX_SPECIES];    /* sigma_s; pair length eps_ij = (sigma_i+sigma_j)/2 */
    float D[CHEMO_MAX_SPECIES];           /* diffusivity D_s, Eq. (1a)/(1b) */
    float chemotactic[CHEMO_MAX_SPECIES]; /* multiplier of chi (Eq. (1b): beta 1, alpha 0) */
    float secrete[CHEMO_MAX_SPECIES];     /* k_s: source k_s rho_s of Eq. (1d) */
    float consume[CHEMO_MAX_SPECIES];     /* kappa_s: sink -kappa_s rho_s c of Eq. (1d) */
    float react_k0[CHEMO_MAX_SPECIES];    /* constant switching rate (r_alpha, Eq. (1c)) */
    float react_kc[CHEMO_MAX_SPECIES];    /* switching rate per unit c (r_beta(c), Eq. (1c)) */
    int32_t react_to[CHEMO_MAX_SPECIES];  /* species a switching cell becomes */
    int32_t reactions;           /* 0 off, 1 fixed-step switching (Sect. 2.1, 3.4) */
    float chi;                   /* chemotactic sensitivity chi, Eq. (1b) */
    float inter;                 /* strength of the soft repulsion (Sect. 3.2) */
    float cutoff_factor;         /* r_c,ij = cutoff_factor * eps_ij (default 1) */
    int32_t cutoff_mode;         /* 0 hard truncation at r_c (as in Sect. 3.2),
                                    1 force shifted to zero at r_c */
    int32_t chem_mode;           /* 0 chemical on the grid (Eq. (1d)),
                                    1 fixed gradient fixed_grad (Sect. 4, c = x) */
    float fixed_grad[3];
    int32_t grid[3];             /* nodes per axis (>= 3); nodes at lo + k h with
                                    h = L/(N-1) (walls) or L/N (periodic) */
    float Dc, gamma;             /* chemical diffusivity and decay, Eq. (1d) */
    int32_t pde_bc;              /* 0 Neumann / no flux (mirror ghost nodes),
                                    1 Dirichlet (wall nodes held), 2 periodic */
    int32_t pde_substeps;        /* 0 = automatic: s = ceil(sum_a 2 Dc dt/h_a^2 / 0.9) */
    double dt;                   /* time step */
    uint64_t seed;               /* Philox4x32-10 key (seed lo, seed hi) */
    int32_t track_displacement;  /* keep the unwrapped displacement (Sect. 4, MSD) */
    float bin_side;              /* cell-list bin side (0 = automatic) */
    int32_t search_mode;         /* 0 automatic (= 4), 1 3^d bins of side >= r_c searched
                                    by the warp together, 2 2^d bins of side >= 2 r_c,
                                    3 3^d bins searched by each lane alone, 4 the upper
                                    half of the 3^d window per lane, each pair once and
                                    its term added to both cells (exact integer sums; an
                                    extra launch and 8 bytes per cell and axis). The
                                    results are identical; only the speed differs */
    int32_t bin_order;           /* 0 or 1: row-major bins, x fastest (2, Z-order: ENOTSUP) */
    int32_t pde_overlap;         /* 0 automatic, 1 run the PDE after the particle kernels,
                                    2 run it concurrently with the particle kernel (one
                                    substep only) */
    int32_t warp_runs;           /* search_mode 1: a warp whose 32 cells fall in at most
                                    this many bins searches them together, a sparser warp
                                    searches per lane (0 = 12; 1..32) */
    int32_t move_scheme;         /* 0 Euler-Maruyama (Eq. (2)); 1 tamed Euler (Sect. 3.2):
                                    drift increment dt a / (1 + dt |a|), a the whole drift */
    int32_t hard_sphere;         /* 1: after the move, overlapping pairs (closer than
                                    (sigma_i + sigma_j)/2) are pushed apart along the line of
                                    centres by twice the penetration, split D_i/(D_i+D_j)
                                    (Sect. 3.2), then the boundary rule again */
    int32_t deposit_kernel;      /* 0 cloud-in-cell (Sect. 2.3); 1 Gaussian kernel density
                                    estimate with bandwidth sigma_s gathered at every node
                                    (Sect. 2.3), truncated at kde_range bandwidths */
    float kde_range;             /* KDE truncation radius in bandwidths (0 = 3) */
    int32_t block_threads;       /* threads per block of the half-window pair kernel and the
                                    move kernel after it: 0 = automatic (256), 128, 256 or 512
                                    (the same registers per thread; chemo_autotune tries them).
                                    Results are identical; only the speed differs */
} chemo_params;

/* Layout facts of a simulation (read-only). */
typedef struct chemo_info {
    int64_t n;                   /* particles */
    int32_t dim;
    int32_t search_mode;         /* 1, 2, 3 or 4, as resolved */
    int32_t nbins[3];            /* bins per axis */
    int64_t bin_slots;           /* entries of the bin table: pitch * nbins[1] * nbins[2] */
    float bin_side[3];
    int32_t bin_pitch;           /* bins per stored row (nbins[0] rounded up to 8); bin
                                    (x, y, z) has key x + pitch (y + nbins[1] z) */
    int32_t pde_substeps;        /* as resolved */
    int64_t grid_nodes;
    int64_t device_bytes;        /* device memory held by the simulation */
    int32_t launches_per_step;   /* kernels one chemo_step launches */
    int32_t layers;              /* replicates stacked in the simulation (1 unless
                                    created by chemo_create_batch) */
    float step_ratio;            /* the time-step rule of thumb (Sect. 3.2): the largest
                                    sqrt(2 (D_i + D_j) dt) / eps_ij over species pairs
                                    with eps_ij > 0 (0 if none). Above 1 a step moves
                                    cells farther than the interaction range; this is
                                    a warning, not an error */
} chemo_info;

typedef struct chemo_sim chemo_sim;

/* Creates a simulation of n cells. pos: n x dim float32 positions (inside
 * the box), species: n uint8 values < n_species; both in memory of mem_kind.
 * Particle ids are 0..n-1 in input order; the Philox counter of a cell is
 * (id, step lo, stream tag, step hi). The chemical field starts at 0 (set it
 * with chemo_write_field). n = 0 is allowed. On success *out receives the
 * handle; release it with chemo_destroy. Errors: EINVAL (bad parameters:
 * dim, species, grid < 3 nodes, periodic box narrower than 2 r_c, more than
 * 2^29 particles...), ENOMEM, ECUDA. */
int chemo_create(const chemo_params *params, int64_t n, const float *pos, const uint8_t *species,
                 int mem_kind, void *stream, chemo_sim **out);

/* Creates an ensemble of `replicates` independent 2D simulations of the same
 * model in one object (the realisations over which the paper averages its
 * statistics, Sect. 4, Fig. 1): replicate r holds n_per_replicate[r] cells
 * (any sizes, 0 allowed), its own copy of the grid, and the Philox key
 * params->seed + r; its cells are ids 0..n_r-1 of that replicate, so replicate
 * r evolves exactly like a chemo_create simulation of its own cells with seed
 * params->seed + r (bitwise for the particles; the field's float atomics may
 * round differently). Caller arrays are the replicates' arrays concatenated in
 * replicate order: pos (sum n_r) x 2, species (sum n_r); grids are
 * replicates x grid[1] x grid[0] (C-order). One chemo_step advances every
 * replicate with the same number of launches as a single simulation.
 * n_per_replicate is host memory. Every other call (write/read state and
 * field, step, step_n, check, stage calls) works on the concatenated arrays;
 * chemo_record / chemo_gradient return ENOTSUP for replicates > 1.
 * Errors: EINVAL (dim != 2 with replicates > 1, replicates < 1 or > 65535, a
 * negative size, more than 2^29 cells in total, the checks of chemo_create),
 * ENOMEM, ECUDA. */
int chemo_create_batch(const chemo_params *params, int32_t replicates, const int64_t *n_per_replicate,
                       const float *pos, const uint8_t *species, int mem_kind, void *stream, chemo_sim **out);

/* Autotuner of the cell list and launch sequence (no counterpart in the
 * paper, which leaves the bin size to the user, Sect. 3.1). Times
 * `trial_steps` steps (after 4 warm-up steps) of the given (batched) particle
 * set for each candidate: search_mode 1 (3^d bins, side r_c x {1, 1.25, 1.5,
 * 2}), 2 (2^d bins, side 2 r_c x {1, 1.25}), 3 (3^d per lane, side r_c x
 * {1, 1.5}) and 4 (half window, side r_c x {1, 1.25, 1.5}), then for mode 1
 * warp_runs {4, 8, 32}, then the PDE overlap on
 * and off; the results do not depend on the choice. *best_out receives
 * params with bin_side, search_mode, warp_runs and pde_overlap set to the
 * fastest candidate, *best_ms_out (if non-NULL) its device time per step.
 * Temporary simulations are created and destroyed on `stream`.
 * Errors: as chemo_create_batch; EINVAL if trial_steps < 1. */
int chemo_autotune(const chemo_params *params, int32_t replicates, const int64_t *n_per_replicate,
                   const float *pos, const uint8_t *species, int mem_kind, int32_t trial_steps, void *stream,
                   chemo_params *best_out, float *best_ms_out);

/* Replaces the particle state: pos (n x dim), species (n) and, if the
 * simulation tracks it, disp (n x dim, NULL = zero). Ids are the array
 * indices. The step index is kept. */
int chemo_write_state(chemo_sim *sim, const float *pos, const uint8_t *species, const float *disp,
                      int mem_kind, void *stream);

/* Replaces the chemical field c (grid_nodes float32, C-order). EINVAL if the
 * simulation has no grid (chem_mode 1). */
int chemo_write_field(chemo_sim *sim, const float *c, int mem_kind, void *stream);

/* Advances one step dt (rows a1-a7 above) on stream. */
int chemo_step(chemo_sim *sim, void *stream);

/* Advances nsteps steps; the result equals nsteps calls of chemo_step. The
 * steps are replayed from a CUDA graph captured on first use. */
int chemo_step_n(chemo_sim *sim, int64_t nsteps, void *stream);

/* Copies the state out by particle id: pos_out (n x dim), species_out (n),
 * disp_out (n x dim; EINVAL if not tracked). Any output may be NULL.
 * Synchronises `stream` when mem_kind is HOST and reports latched device
 * errors. */
int chemo_read_state(chemo_sim *sim, float *pos_out, uint8_t *species_out, float *disp_out,
                     int mem_kind, void *stream);

/* Copies the chemical field c^n out (grid_nodes float32, C-order). */
int chemo_read_field(chemo_sim *sim, float *c_out, int mem_kind, void *stream);

/* Records a run for the adjoint: advances nsteps steps exactly like
 * chemo_step_n (same kernels, same Philox counters) while keeping checkpoints
 * of the state and the field every `every` steps in library memory (replacing
 * any earlier recording). The adjoint covers the model without type switching
 * and without consumption, with Neumann or periodic fields: ENOTSUP
 * otherwise. */
int chemo_record(chemo_sim *sim, int64_t nsteps, int32_t every, void *stream);

/* chemo_record that also keeps, during the run, the states the reverse sweep
 * reads (positions, fields, sorted states with their cell lists, pair
 * forces) for the latest segments that fit in store_bytes of device memory
 * (store_bytes < 0: every segment; 0: none, which is chemo_record). The
 * gradient re-runs only the other segments, so with every segment stored it
 * is the reverse sweep alone. The checkpoints are taken as in chemo_record.
 * A stored segment is stepped launch by launch (no graph replay). Memory per
 * stored segment: every x (n x (8 d + 16) + 4 grid_nodes + 4 x the cell
 * list's words) bytes, plus n x 4 d. Errors: as chemo_record; ENOMEM if the
 * stored segments do not fit. */
int chemo_record_stored(chemo_sim *sim, int64_t nsteps, int32_t every, int64_t store_bytes, void *stream);

/* Vector-Jacobian product (adjoint) of the last recorded run: given
 * dL/dpos of its final state (n x dim by id) and optionally dL/dc of its
 * final field (grid_nodes, NULL = 0), returns dL_dparams = [dL/dchi,
 * dL/dinter, dL/dD_0 .. dL/dD_{n_species-1}] and, if dL_dpos0 is non-NULL,
 * dL/dpos of the recorded run's initial state. The noise is frozen (the same
 * Philox counters as the forward run); each segment between checkpoints is
 * re-run forward before its reverse sweep, the re-run of the segment before
 * it overlapping that sweep on a second stream (Sect. 2 model: pair force Jacobian,
 * interpolation Jacobian, reflection signs, deposit and PDE transposes). The
 * cutoff jump and the reflection kinks are not differentiated (measure-zero
 * events). dL/dinter is 0 when inter = 0 (no pair force, no cell list for
 * its cutoff). Memory: two segments' states, fields, sorted states, cell
 * lists and pair forces of `every` steps each (segments kept by
 * chemo_record_stored are not re-run). The simulation is left at the final
 * state and step index of the recorded run, whatever was stepped after the
 * record. An ensemble (chemo_create_batch) is differentiated as a whole: its
 * replicates share the parameters, so dL_dparams is the sum of every
 * replicate's part, and positions are by the ids of the batch. Synchronises
 * `stream` when mem_kind is HOST. EINVAL if no run is recorded. */
int chemo_gradient(chemo_sim *sim, const float *dL_dpos_final, const float *dL_dc_final, float *dL_dparams,
                   float *dL_dpos0, int mem_kind, void *stream);

/* Replaces the model parameters of a live simulation. Geometry (dim, box,
 * grid, boundary, species count, bin layout) must not change: EINVAL. */
int chemo_set_params(chemo_sim *sim, const chemo_params *params);

/* Absolute index of the next step (0 after create). */
int64_t chemo_step_index(const chemo_sim *sim);

/* Sets the absolute step index (the Philox counter of the next step). */
int chemo_set_step_index(chemo_sim *sim, int64_t step, void *stream);

/* Synchronises stream and returns the first latched device error, then
 * clears it. */
int chemo_check(chemo_sim *sim, void *stream);

/* Failure-detection test of the one device-side wait (the look-back of the
 * cell-list scan, a decoupled look-back after Merrill & Garland; no
 * counterpart in the paper). Runs one scan of the simulation's idle count
 * buffer with its tile counter started at 1 instead of 0, so no block
 * claims tile 0 and the tiles after it wait on a predecessor that never
 * publishes; each wait gives up after spin_limit polls (the library's own
 * scans use 2^22, about 0.1 s) and latches CHEMO_ETIMEOUT, which the next
 * chemo_check returns and clears. The offsets go to scratch memory and the
 * scan's counters are reset afterwards, so the simulation's state and cell
 * list are untouched and the next step is a normal one. Asynchronous on
 * `stream`. EINVAL for spin_limit 0 or a cell list of a single scan tile
 * (4096 groups of 8 bins or fewer), where no tile waits on another. */
int chemo_stall_scan(chemo_sim *sim, uint32_t spin_limit, void *stream);

/* Fills *info. */
int chemo_get_info(const chemo_sim *sim, chemo_info *info);

/* Measurement: advances nsteps steps exactly like chemo_step (same kernels,
 * same streams and overlap), with a CUDA event pair around every kernel on
 * the stream it runs on. Returns in kernel_ms[CHEMO_PROF_SLOTS]: the mean
 * device time (ms) per step of the particle kernel, the PDE (all substeps),
 * the scan, the scatter + deposit, and of a whole step; then the mean number
 * of in-cutoff pair interactions per step (each ordered pair counted once
 * per cell) and the mean number of candidate distance tests per step of the
 * half-window search (0 for the other searches). Synchronises `stream`. */
#define CHEMO_PROF_SLOTS 7
int chemo_profile_steps(chemo_sim *sim, int64_t nsteps, float *kernel_ms, void *stream);

/* Observables of the current state, reduced on the device (the statistics
 * of Sect. 4). out (mem_kind memory) receives, per replicate (1 unless the
 * simulation is a batch), 8 x 5 + 1 doubles: for each species slot s < 8 the
 * number of cells, their mean unwrapped displacement (x, y, z; 0 unless
 * track_displacement) and mean squared displacement, then the chemical mass
 * h^d sum_k tau_k c_k (trapezoid weights tau: 1/2 per wall axis at boundary
 * nodes, 1 on a periodic grid; 0 without a grid). Synchronises `stream` when
 * mem_kind is HOST. */
int chemo_observables(chemo_sim *sim, double *out, int mem_kind, void *stream);

/* Occupancy histogram of the cells: the box cut into shape[0] x shape[1]
 * (x shape[2] in 3D) equal parts (1..4096 per axis); hist_out (mem_kind
 * memory, float32) receives per replicate and species the count of cells in
 * each part, C-order [replicate][species][z][y][x] (exact up to 2^24 per
 * part). Cells on the upper wall count in the last part. Synchronises
 * `stream` when mem_kind is HOST. EINVAL for a bad shape. */
int chemo_histogram(chemo_sim *sim, const int32_t *shape, float *hist_out, int mem_kind, void *stream);

/* Releases every resource of sim (NULL is ignored). Synchronises the device
 * work of the simulation first. */
void chemo_destroy(chemo_sim *sim);

/* Device memory source (plumbing; no counterpart in the paper). Every device
 * buffer of the library (a simulation's state, cell list, grids and scratch,
 * a recorded run's tape, the temporaries of chemo_philox and
 * chemo_init_positions) is allocated once, outside the step, and comes from
 * cudaMalloc unless an allocator is set here. alloc(ctx, bytes, &ptr) returns
 * 0 and a device pointer of the current device aligned to 256 bytes, or
 * non-zero on failure (the call that needed the memory then returns ENOMEM
 * and releases what it had taken); release(ctx, ptr, bytes) takes back a
 * pointer with the size it was allocated with. The library calls release only
 * after the work that used the buffer has finished on the device. Both
 * callbacks are called from the thread of the library call, never inside a
 * stream capture or a kernel. The setting is process-wide and read when a
 * simulation is created (or a temporary is needed): a simulation keeps the
 * allocator it was created with until chemo_destroy. alloc and release are
 * both set or both NULL (NULL, NULL restores cudaMalloc / cudaFree).
 * Errors: EINVAL if exactly one of them is NULL. Touches no GPU. */
typedef int (*chemo_alloc_fn)(void *ctx, size_t bytes, void **ptr);
typedef void (*chemo_release_fn)(void *ctx, void *ptr, size_t bytes);
int chemo_set_allocator(chemo_alloc_fn alloc, chemo_release_fn release, void *ctx);

/* Static text of a status code. */
const char *chemo_status_string(int status);

/* Message of the last failed call on this thread ("" if none). */
const char *chemo_last_error(void);

/* ---------------------------------------------------------------------- */
/* Stage-level entry points. They run the step's own kernels on the current */
/* state without advancing it, so each row of the step can be checked on   */
/* its own. Outputs are indexed by particle id unless stated.              */
/* ---------------------------------------------------------------------- */

/* Raw Philox4x32-10 words (Salmon et al., SC'11) of the device generator:
 * ctr n x 4 uint32, key (seed lo, seed hi), out n x 4 uint32. */
int chemo_philox(uint64_t seed, const uint32_t *ctr, uint32_t *out, int64_t n, int mem_kind,
                 void *stream);

/* Initial state of the paper's experiments (Sect. 3), drawn on the device:
 * cells i < n_alpha are species 0 (alpha), normal around the box centre with
 * standard deviation sigma_frac x the box width per axis (0.1 in the paper),
 * put inside by the box's boundary rule (reflection, or wrap when periodic);
 * cells i >= n_alpha are species 1 (beta), uniform in the box. Cell i uses the
 * Philox4x32-10 words of counter (i, 0, 3, 0) under the key params->seed:
 * Box-Muller on (w0, w1) and (w2, w3) for alpha, u = (w_a + 1/2) 2^-32 per
 * axis for beta. Writes pos_out (n x dim float32) and species_out (n uint8)
 * in memory of mem_kind (HOST: synchronises `stream`). EINVAL for bad sizes,
 * sigma_frac <= 0, or beta cells with n_species < 2. */
int chemo_init_positions(const chemo_params *params, int64_t n, int64_t n_alpha, float sigma_frac, float *pos_out,
                         uint8_t *species_out, int mem_kind, void *stream);

/* Row a1: the bin cell of every particle, n x dim int32 (cell coordinates
 * per axis, not the Morton key). */
int chemo_stage_bins(chemo_sim *sim, int32_t *cells_out, int mem_kind, void *stream);

/* Row a2: the sorted order: ids_out[j] = id of the j-th particle in the
 * sorted (binned) arrays (n uint32), and bin_start_out (bin_slots + 1
 * uint32) the offsets of every bin slot in that order (NULL to skip). */
int chemo_stage_sort(chemo_sim *sim, uint32_t *ids_out, uint32_t *bin_start_out, int mem_kind,
                     void *stream);

/* Row a3: the pair force F_i (n x dim float32), and optionally per particle
 * the number of neighbours inside the cutoff (count_out, n int32) and the
 * sum of their ids (idsum_out, n uint64). */
int chemo_stage_forces(chemo_sim *sim, float *F_out, int32_t *count_out, uint64_t *idsum_out,
                       int mem_kind, void *stream);

/* Row a4: the chemotactic drift chi * chemotactic_s * grad c(X_i) (n x dim). */
int chemo_stage_drift(chemo_sim *sim, float *drift_out, int mem_kind, void *stream);

/* Row a6: the density terms deposited by the current positions on the grid:
 * S_out = dt sum_i k_s w_ik/(tau_k h^d) and R_out = sum_i kappa_s w_ik/(tau_k
 * h^d) (grid_nodes each, C-order; either may be NULL). */
int chemo_stage_deposit(chemo_sim *sim, float *S_out, float *R_out, int mem_kind, void *stream);

/* ---------------------------------------------------------------------- */
/* Slab decomposition of one system along z (sub-domains).                 */
/* ---------------------------------------------------------------------- */

/* One system (3D, reflecting walls, a grid) splits into slabs along z, one
 * sub-domain simulation per slab (on one GPU or one per GPU). The paper runs
 * one domain; these calls are the exchange points of its step (Sect. 3:
 * interaction, move, deposit, PDE) across slab faces:
 *
 *   - a sub-domain holds the cells it owns (z in its slab) and ghosts:
 *     copies of the neighbours' cells within the interaction range of a face
 *     (Sect. 2.2), which add their pair force to owned cells and are neither
 *     moved nor deposited (their owner does both);
 *   - its box and grid are the slab widened by halo planes of the global
 *     grid; an inner face (open) does not reflect, so an owned cell may step
 *     into the halo and then migrates to the neighbour;
 *   - deposits of owned cells onto halo planes are added to the neighbour's
 *     source before its PDE (chemo_slab_planes, op ADD), and after the PDE the
 *     halo planes of c are refreshed from the neighbours (op WRITE).
 *
 * Per step: chemo_step_particles on every sub-domain; fold the halo planes of
 * the source and consumption grids into the neighbours; chemo_step_field;
 * refresh the halo planes of c; chemo_slab_select into the cell sets of the
 * sub-domain and its two neighbours; chemo_slab_ingest of each sub-domain's
 * own set and the two it received. The noise is keyed by the cells' ids,
 * which travel with them, so the decomposed run takes the steps of the
 * single-domain run; results differ from it only by the order of the float
 * additions of the deposit and the rounding of a sub-domain's grid origin. */

#define CHEMO_OPEN_ZLO 1u           /* open_faces bit: the z = lo face is an inner face */
#define CHEMO_OPEN_ZHI 2u           /* open_faces bit: the z = hi face is an inner face */
#define CHEMO_GHOST_ID 0x1FFFFFFFu  /* id of a ghost cell in chemo_cell.tag */

/* One cell in transit between sub-domains: 32 bytes, arrays of them 16-byte
 * aligned. tag = id | species << 29 (id < CHEMO_GHOST_ID, or CHEMO_GHOST_ID
 * for a ghost); (dx, dy, dz) is the displacement since the run began (zero
 * unless the simulation tracks it). */
typedef struct chemo_cell {
    float x, y, z;
    uint32_t tag;
    float dx, dy, dz;
    uint32_t reserved;
} chemo_cell;

/* Destination of chemo_slab_select: the cells with z0 <= z < z1 are
 * appended to out (device memory, `capacity` records); those outside
 * own0 <= z < own1 are written as ghosts. count points to two device
 * counters that the call adds to: [0] cells selected, [1] of them owned
 * (not ghosts). Cells past capacity are counted but not written, so
 * count[0] > capacity reports an overflow. */
typedef struct chemo_slab_target {
    float z0, z1, own0, own1;
    chemo_cell *out;
    int64_t capacity;
    unsigned long long *count;
} chemo_slab_target;

/* An empty sub-domain. params describes the slab with its halo: the box's z
 * extent and grid[2] are those of the halo-widened slab, cut from the global
 * grid at node planes (node spacing as in the global grid), every other
 * field as for the whole system. Needs dim 3, boundary 0 (walls), chem_mode
 * 0 and none of hard_sphere, deposit_kernel 1; pde_bc 0 or 1. capacity >= 1
 * is the most cells (owned and ghosts) it will hold; open_faces is a mask of
 * CHEMO_OPEN_ZLO / CHEMO_OPEN_ZHI. The deposit always goes to the source
 * and consumption grids (read by chemo_slab_planes grids 1 and 2), the PDE
 * runs after it on one stream. A move that leaves the box through an open
 * face is clamped and latched as CHEMO_EDOMAIN (the halo was too thin).
 * chemo_read_state, chemo_write_state, chemo_record*, chemo_observables,
 * chemo_histogram and the stage calls return CHEMO_ENOTSUP for sub-domains
 * (read cells with chemo_slab_select; the field with chemo_read_field or
 * chemo_slab_planes). */
int chemo_create_subdomain(const chemo_params *params, int64_t capacity, uint32_t open_faces, void *stream,
                           chemo_sim **out);

/* Replaces the cells of a sub-domain by n records (0 <= n <= capacity,
 * host or device memory as mem_kind; device arrays 16-byte aligned) and
 * bins them; the field, the step index and the source grids are kept.
 * Positions outside the box are clamped and latched (CHEMO_EDOMAIN), species
 * out of range taken as 0 and latched. */
int chemo_slab_ingest(chemo_sim *sim, int64_t n, const chemo_cell *cells, int mem_kind, void *stream);

/* Appends the sub-domain's own (non-ghost) cells to up to 4 targets (each
 * cell to every target whose [z0, z1) holds it), asynchronously on stream;
 * targets is host memory read during the call. */
int chemo_slab_select(chemo_sim *sim, int32_t ntargets, const chemo_slab_target *targets, void *stream);

/* Planes plane0 .. plane0 + nplanes - 1 (z index of the sub-domain's grid;
 * g[0] x g[1] floats each, C-order) of grid 0 (c, the current field), 1 (the
 * source S deposited since the last field step) or 2 (the consumption rate R
 * deposited since then), against buf (device memory of at least
 * nplanes x g[1] x g[0] floats; the call cannot check its size):
 * op 0 reads the planes into buf, 1 writes buf into them, 2 adds buf to
 * them. Asynchronous on stream. */
#define CHEMO_PLANES_READ 0
#define CHEMO_PLANES_WRITE 1
#define CHEMO_PLANES_ADD 2
int chemo_slab_planes(chemo_sim *sim, int32_t grid, int32_t op, int64_t plane0, int64_t nplanes, float *buf,
                      void *stream);

/* The two halves of chemo_step on a sub-domain: chemo_step_particles runs
 * rows a1-a6 (pair force, drift, move, re-binning, deposit into the source
 * grids, which it clears first) and advances the step index;
 * chemo_step_field runs row a7 (the PDE substeps, reading the source grids).
 * chemo_step on a sub-domain runs both with no exchange between them.
 * CHEMO_ENOTSUP for other simulations. */
int chemo_step_particles(chemo_sim *sim, void *stream);
int chemo_step_field(chemo_sim *sim, void *stream);

/* ---------------------------------------------------------------------- */
/* Pair forces without device allocation.                                  */
/* ---------------------------------------------------------------------- */

/* Row a3 (the pair force F_i, n x dim float32 by particle index) of a
 * caller's particle set, computed without allocating any device memory. The
 * paper has no counterpart; this entry point exists for callers that cannot
 * call cudaMalloc where they need forces: applications that give the library
 * a fixed device-memory budget at start-up, real-time loops in which an
 * allocation (which can synchronise the device) would break the timing, and
 * plug-ins running inside another framework's memory manager.
 *
 * pos (n x dim float32), species (n uint8) and F_out must be device memory;
 * params as for chemo_create (only the geometry, species and force fields
 * matter). The cell list is built in one static device array owned by the
 * library (about 3.4 MB, held on every GPU that loads the library until the
 * process exits), so: n <= 65535 (the largest 16-bit bin count, so that no
 * bin can overflow even with every particle in it) and the cell list may use
 * at most 262144 bins, else CHEMO_EINVAL with a message naming the limit.
 * All calls share the array and it keeps the last call's contents; calls
 * whose kernels overlap on the GPU (different streams without ordering) race
 * on it. The first call on a device looks up the array's device address,
 * with that device current; make that first call before any stream capture.
 * The call is asynchronous on `stream` and returns before the kernels run,
 * so conditions found on the device are not reported: a non-finite
 * coordinate (taken as the box's lower bound on that axis), a species out of
 * range (taken as species 0), a position outside the box (clamped to the
 * box) and a bounded wait of the cell-list scan that ran out (possible only
 * when other work starves the kernel; the forces are then unspecified).
 * Validate inputs on the host where these can occur. */
int chemo_forces_noalloc(const chemo_params *params, int64_t n, const float *pos, const uint8_t *species,
                         float *F_out, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* CHEMO_H */
