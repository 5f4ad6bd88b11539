/*
 * flexrt.h -- C ABI of libflexrt: the adaptive ray-tracing radiative-transfer
 * step of FlexRT (Cain & D'Aloisio, arXiv:2409.04521) on one GB300 GPU.
 *
 * One call to flexrt_step() advances a simulation by one RT step, in the
 * order the paper states it:
 *   1. emission:  every source cell casts 12*4^l_src rays from its centre along
 *                 the NESTED HEALPix pixel centres of a sphere that is randomly
 *                 rotated each step (Sec. 3.1, Eq. 1);
 *   2. march:     every ray moves exactly one cell width and is attenuated by
 *                 exp(-tau), tau = kappa * ds, kappa = n_HI sigma_nu + 1/lambda_mfp
 *                 (Sec. 3.1; Sec. 4.2, Eq. 13);
 *   3. deposit:   absorbed photons go to the crossed cells as the finite-mfp
 *                 photo-ionisation rate of Sec. 4.2, Eq. 17 (which reduces to
 *                 Eq. 5 when lambda = 1/(n_HI sigma));
 *   4. split:     a level-l ray that has travelled r_split(l) (Sec. 3.2, Eq. 2)
 *                 becomes the four rays (l+1, 4p+i) (Eq. 3);
 *   5. merge:     optional (flexrt_options.merge): the floor(N_ex * N_RT)
 *                 brightest rays are exempt; the others merge per (cell, pixel
 *                 of a randomly oriented level-l_merge HEALPix sphere of that
 *                 cell) into one ray along the pixel centre (Sec. 3.3, Eq. 4);
 *   6. chemistry: per cell, the time-dependent ionisation update of Sec. 4.1,
 *                 Eq. 7-10, and the temperature equation Eq. 12.
 *
 * Conventions for every entry point:
 *   - host pointers are read during the call and never kept; output buffers
 *     are caller-owned host memory;
 *   - no C++ exception crosses the ABI; every call returns flexrt_status and
 *     the context keeps a message for flexrt_last_error();
 *   - a context is used by one host thread at a time; its device work runs on
 *     the CUDA stream given in flexrt_options.cuda_stream (0 = a stream the
 *     library creates);
 *   - flexrt_step() only enqueues work.  Device-side failures (ray-queue
 *     overflow) are latched: the failed step leaves the state of the last good
 *     step, later steps do nothing, and the status is returned by the next
 *     flexrt_step() or flexrt_sync() that sees it; the getters keep returning
 *     the state of the last good step.
 *   - device memory is allocated by flexrt_create (cells, ray queues) and by
 *     flexrt_add_sources (emitter tables, when they grow), and freed by
 *     flexrt_destroy; the probes allocate and free their own scratch.
 */
#ifndef FLEXRT_H
#define FLEXRT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    FLEXRT_OK = 0,
    FLEXRT_E_INVALID = 1,   /* bad argument                                  */
    FLEXRT_E_OOM = 2,       /* device or host allocation failed              */
    FLEXRT_E_CAPACITY = 3,  /* ray queue, emitter or cell arena full         */
    FLEXRT_E_CUDA = 4,      /* CUDA runtime error                            */
    FLEXRT_E_TIMEOUT = 5,   /* reserved: no call waits on the device with a limit */
    FLEXRT_E_STATE = 6      /* call not valid in the current state           */
} flexrt_status;

#define FLEXRT_MAX_BINS 8
#define FLEXRT_MAX_LEVEL 12

typedef struct flexrt_ctx flexrt_ctx;
typedef struct flexrt_batch flexrt_batch;

/* Uniform Cartesian grid of cubic RT cells, x fastest in every cell array. */
typedef struct { int32_t nx, ny, nz; } flexrt_grid;

/* Box: comoving length of the x side in cm and the (fixed) redshift.  The
 * physical cell width is box_cm_comoving / nx / (1 + redshift). */
typedef struct { double box_cm_comoving; double redshift; } flexrt_box;

/* Spectrum in nbins frequency bins (Sec. 4.1, Eq. 5 sums over them):
 * frac[b]      fraction of a source's photons in bin b (sum 1),
 * sigma_cm2[b] HI photo-ionisation cross-section of bin b,
 * eheat_erg[b] mean energy above 13.6 eV given to the gas per ionisation. */
typedef struct {
    int32_t nbins;
    const double *frac, *sigma_cm2, *eheat_erg;
} flexrt_spectrum;

/* Sub-grid opacity, the 1/lambda_mfp term of kappa (Sec. 4.2, Eq. 13, 15):
 * mode 0: none; mode 1: constant comoving lambda0 everywhere;
 * mode 2: in cells with x_HII >= xion_threshold,
 *   lambda = lambda0 * Delta^-delta_exp * (max(Gamma, gamma_floor)/gamma_ref)^gamma_exp
 *   with Delta = n_H / nH_mean (nH_mean = 0: mean of the grid) and Gamma the
 *   previous step's rate (in Generalized mode: the ionised part of every
 *   lit cell);
 * mode 3 (Generalized mode only): photo-ionisation equilibrium in the
 *   ionised part, n_HI = alpha_B (1 + chi) n_H^2 / max(Gamma, gamma_floor),
 *   kappa_nu = sigma_nu n_HI (Sec. 5.1, Eq. 20-22).  A part not lit yet is
 *   optically thin (Eq. 14). */
typedef struct {
    int32_t mode;
    double lambda0_cm_comoving, delta_exp, gamma_ref, gamma_exp, gamma_floor,
        xion_threshold, nH_mean;
} flexrt_mfp;

typedef struct {
    int32_t l_src;          /* HEALPix level of emission (Eq. 1)                */
    int32_t l_max;          /* deepest split level, <= FLEXRT_MAX_LEVEL         */
    double n_ray_min;       /* N_ray^min of Eq. 2                              */
    double eps_term;        /* ray dropped below eps * its unattenuated content */
    uint64_t seed;          /* seed of the per-step sphere rotations            */
    int32_t rotate;         /* 1: rotate each sphere each step (Sec. 3.1)       */
    int32_t isothermal;     /* 1: T fixed; 0: Eq. 12                            */
    int32_t rates;          /* 0: constant alpha_B, no collisional ionisation;
                               1: temperature-dependent rate fits               */
    int32_t chem_iters;     /* n_e re-evaluations of Eq. 7-10 per step          */
    double alpha_B_const;   /* cm^3/s, used when rates == 0                     */
    double x_init, T_init;  /* initial ionised fraction and temperature (K)     */
    int64_t ray_capacity;   /* live rays a queue holds (slots allocated: 1.25x
                               plus 4096); 0 = sized from free memory         */
    int32_t keep_diagnostics; /* 1: keep per-cell segment counts of each step   */
    void *cuda_stream;      /* cudaStream_t, 0 = library-owned stream           */
    /* Ray merging at the end of every step (Sec. 3.3, Eq. 4).  A merged ray
     * points along the centre of its merge pixel; its position, distance
     * travelled and HEALPix level are the photon-weighted means of its
     * constituents' (level at least l_merge), its photons their sum.  Until it
     * splits it stands for the four level-(l+1) pixels around that centre. */
    int32_t merge;          /* 1: merge rays                                    */
    int32_t l_merge;        /* merge-sphere level, 0..min(11, l_max)            */
    double n_ex;            /* rays per RT cell exempt from merging (N_ex)      */
    /* Passes of the Gamma - <n_HI> iteration (Sec. 4.1, Eq. 7-11; with the
     * sub-grid law also lambda - Gamma, Sec. 4.2): each pass re-marches the
     * step from the same start with the opacity of the previous pass's
     * time-averaged neutral fraction (and its Gamma in lambda); the last pass
     * is committed.  1 = one pass with the start-of-step opacity.  Members of
     * a batch must all use the same value. */
    int32_t gamma_iters;
    /* Generalized Opacity mode (Sec. 4.2, Eq. 14-22): a cell is a highly
     * ionised fraction x_ion, crossed with the sub-grid opacity of its mfp
     * law, and a neutral rest behind an infinitely thin screen that absorbs
     * what reaches it and advances (Eq. 18-19); chemistry is the cell's atom
     * balance instead of Eq. 7-10.  Needs gamma_iters >= 4: lambda, Gamma
     * and each screen's share of the photons reaching it are iterated towards
     * self-consistency.  A screen's share comes from the previous pass; a
     * screen first reached in the last pass absorbs all that reaches it, and
     * what exceeds its atoms is lost (counted as absorbed): on a 32^3
     * Stromgren sphere's first 40 steps 8e-3 of the emitted photons with 3
     * passes, 2e-3 with 4, 2e-6 with 5 (how fast the cascade of newly
     * reached screens settles depends on the random spheres).  chi: He/H number ratio, singly
     * ionised helium in Eq. 18.
     * With isothermal = 0 the ionised part's temperature evolves: gas that
     * ionises enters at t_reion (K; 0 < t_reion < 1e9, -1 < alpha_pl < 20;
     * E_INVALID otherwise) and mixes by mass with the gas ionised before;
     * then Eq. 12 at static density with the photo-heating of Eq. 22
     * (power-law spectrum of index alpha_pl cut at 4 Ryd, case-A
     * recombinations balanced by ionisations) against the cooling rates, with
     * n_HI from the ionised part's neutral fraction.  Gas the screen has not
     * reached keeps its temperature (no pre-heating). */
    int32_t gen_mode;
    double chi;
    double t_reion;
    double alpha_pl;
    /* Cap on the device memory the context allocates (bytes; 0 = none).  An
     * allocation that would pass it fails as if the device were full:
     * flexrt_create returns FLEXRT_E_OOM, frees whatever it had allocated
     * and leaves *out NULL; flexrt_add_sources returns FLEXRT_E_OOM and the
     * context keeps its previous sources. */
    int64_t device_bytes_max;
} flexrt_options;

/* Fill *o with defaults (l_src 0, l_max 12, N_min 3, eps 1e-10, seed 1,
 * rotate 1, isothermal 1, rates 0, 5 iterations, alpha_B 2.59e-13,
 * x_init 1.2e-3, T_init 1e4, automatic capacity, library stream, no merging,
 * l_merge 0, N_ex 16, one pass per step, Standard mode, chi 0,
 * t_reion 2e4 K, alpha_pl 1.5). */
void flexrt_default_options(flexrt_options *o);

/* Create one simulation.  n_H: host, nx*ny*nz doubles, physical cm^-3,
 * x fastest.  Copies every input to the device.  *out receives the context. */
flexrt_status flexrt_create(const flexrt_grid *grid, const flexrt_box *box,
                            const double *n_H, const flexrt_mfp *mfp,
                            const flexrt_spectrum *spectrum,
                            const flexrt_options *opt, flexrt_ctx **out);

/* Add n point sources: cell_ijk host int32[3n] (i,j,k), ndot host double[n]
 * photons/s.  Sources sharing a cell form one emitter (Sec. 3.1: rays are cast
 * from each cell that holds sources) whose rate is their sum; emitters are
 * numbered in order of first appearance. */
flexrt_status flexrt_add_sources(flexrt_ctx *ctx, int32_t n, const int32_t *cell_ijk,
                                 const double *ndot);

/* Enqueue one RT step of length dt_s seconds (asynchronous). */
flexrt_status flexrt_step(flexrt_ctx *ctx, double dt_s);

/* The same step in two stages, for inspecting the rays the merge takes
 * (diagnostics): stage 1 enqueues the emission and the marches of the step
 * of length dt_s; stage 2 (dt_s ignored) the merge, the chemistry and the
 * commit.  Between the two, flexrt_get_rays and flexrt_get_rays_merged
 * return the march's output, before merging; flexrt_step, the checkpoint
 * calls and another stage 1 return FLEXRT_E_STATE. */
flexrt_status flexrt_step_stage(flexrt_ctx *ctx, double dt_s, int32_t stage);

/* Wait for all enqueued work; returns a latched device error if any.  No
 * call of this library waits on the device with a time limit, so
 * FLEXRT_E_TIMEOUT is reserved and never returned. */
flexrt_status flexrt_sync(flexrt_ctx *ctx);

/* Restore the state right after flexrt_create + flexrt_add_sources (fields,
 * rays, step counter, photon budget) without touching host memory. */
flexrt_status flexrt_reset(flexrt_ctx *ctx);

/* Per-cell fields after the last step, host doubles (NULL = skip):
 * gamma_HI (1/s, Eq. 17), x_HII, T (K), n_HI (cm^-3). Synchronises. */
typedef struct { double *gamma_HI, *x_HII, *T, *n_HI; } flexrt_fields;
flexrt_status flexrt_get_fields(flexrt_ctx *ctx, flexrt_fields *f);

/* Photon budget in photons: out[0] emitted, out[1] absorbed (sum over cells
 * of deposited photons), out[2] escaped through the box faces, out[3] in
 * flight in live rays.  emitted = absorbed + escaped + in flight. */
flexrt_status flexrt_get_budget(flexrt_ctx *ctx, double out[4]);

/* Generalized Opacity mode (Sec. 4.2, Eq. 18): photons that moving screens
 * absorbed beyond the neutral atoms their cells had, since creation/reset --
 * part of out[1] of flexrt_get_budget that ionised nothing (a screen first
 * reached in the step's last pass of the Gamma - <n_HI> iteration takes all
 * that reaches it; more passes shrink it).  0 in Standard mode. */
flexrt_status flexrt_get_screen_excess(flexrt_ctx *ctx, double *photons);

/* Counters: out[0] live rays, out[1] ray-cell segments of the last step,
 * out[2] segments since creation/reset, out[3] steps taken, out[4] queue
 * capacity, out[5] rays marched in the last step. */
flexrt_status flexrt_get_counts(flexrt_ctx *ctx, int64_t out[6]);

/* Diagnostics (need keep_diagnostics = 1): ray-cell segments per cell in
 * the last step, host int32[ncell]. */
flexrt_status flexrt_get_segment_counts(flexrt_ctx *ctx, int32_t *out);

/* Diagnostics: copy up to cap live rays to host arrays (NULL = skip):
 * level, pixel (NESTED), emitter, birth step, direction int32[3] (2^-21 cell
 * per step), photons double[nbins] (photons, physical).  *n gets the count. */
flexrt_status flexrt_get_rays(flexrt_ctx *ctx, int64_t cap, int32_t *level, int64_t *pixel,
                              int32_t *emitter, int32_t *birth, int32_t *dir, double *photons,
                              int64_t *n);
/* Generalized mode: the highly ionised volume fraction x_ion per cell, host
 * doubles[ncell] (0 for a Standard-mode simulation).  Synchronises. */
flexrt_status flexrt_get_ionized_volume(flexrt_ctx *ctx, double *x_ion);

/* For a ray made by a merge, flexrt_get_rays reports emitter = -1 - (local
 * index of the cell it was merged in), birth = the step of the merge and
 * pixel = its merge pixel (a vertex ray) or its NESTED pixel after splits.
 * The same rays in the same order (NULL = skip): merged int32[n] (1 for a
 * merged ray or a split child of one), vertex int32[n] (1: an unsplit merged
 * ray of level above l_merge), dist int32[n] (cells travelled at the merge),
 * pos int64[3n] (position at the merge, 2^-21 cell), thr double[n]
 * (termination threshold, photons). */
flexrt_status flexrt_get_rays_merged(flexrt_ctx *ctx, int64_t cap, int32_t *merged, int32_t *vertex,
                                     int32_t *dist, int64_t *pos, double *thr, int64_t *n);

/* Checkpoint and restart (no counterpart in the paper: a facility for long
 * runs).  flexrt_save_state writes the state a later step reads -- per-cell
 * neutral fraction, ionised fraction, temperature, Gamma, opacity and
 * Generalized-mode state, the live rays, the emitters' photons per ray and
 * rotation ring, the step counter, dt and the photon budget -- into the
 * caller's host buffer buf of cap bytes; with buf == NULL it only stores the
 * size needed in *bytes (FLEXRT_E_CAPACITY if cap is too small).  It waits
 * for enqueued work.  flexrt_load_state restores such a buffer into a
 * context created with the same grid, spectrum bins, sources, queue layout
 * (merging on or off) and a ray capacity that holds its rays; FLEXRT_E_INVALID
 * for a buffer of another simulation, with the context unchanged.  A restored
 * context continues exactly as the saved one would: the next step marches the
 * same rays through the same opacities.  Options (N_ex, passes ...) are those
 * of the context it is loaded into. */
flexrt_status flexrt_save_state(flexrt_ctx *ctx, void *buf, int64_t cap, int64_t *bytes);
flexrt_status flexrt_load_state(flexrt_ctx *ctx, const void *buf, int64_t bytes);

/* Device memory the context has allocated, in bytes (the quantity
 * flexrt_options.device_bytes_max caps). */
flexrt_status flexrt_get_device_bytes(flexrt_ctx *ctx, int64_t *bytes);

/* Per-kernel device time accumulated since the last call (CUDA events on
 * the context stream): "emit", "march", "chem" and "merge" (all kernels of
 * the merge step); ms[k], launches[k].  Timing is only recorded when enabled
 * by flexrt_profile(ctx, 1). */
flexrt_status flexrt_profile(flexrt_ctx *ctx, int32_t enable);
flexrt_status flexrt_get_kernel_times(flexrt_ctx *ctx, double ms[4], int64_t launches[4],
                                      int64_t march_rays[1]);

/* Launch configuration of the fused march kernel (chosen by the autotuner):
 * agg: how lanes of a warp combine deposits into one cell before the
 * vector reduction (0 none, 1 groups of equal cells, 2 runs of equal
 * consecutive cells); minb: resident blocks per SM the register budget
 * targets (2..4); blocks_per_sm: persistent blocks launched per SM
 * (0 = occupancy limit); threads: threads per block, 128 or 256 (0 = 256);
 * slab: queue slots a warp reserves for its output at a time, 32..4096
 * (0 = 512).  FLEXRT_E_INVALID if the variant is not built or a value is
 * out of range. */
flexrt_status flexrt_set_launch(flexrt_ctx *ctx, int32_t agg, int32_t minb, int32_t blocks_per_sm,
                                int32_t threads, int32_t slab);

/* Message of the context's last failure; with ctx == NULL, of the last failed
 * call without a context (probes) on this host thread. */
const char *flexrt_last_error(const flexrt_ctx *ctx);
void flexrt_destroy(flexrt_ctx *ctx);

/* ----------------------------------------------------------------------- */
/* Device-function probes.  Each runs the very device function the step    */
/* kernels use, on host inputs, and returns host outputs.  Synchronous.     */
/* ----------------------------------------------------------------------- */

/* Fixed-point NESTED HEALPix vectors (Sec. 3.1): for pixels p0..p0+n-1 of
 * `level`, out int32[3n] = round(v * 2^24). */
flexrt_status flexrt_probe_pixvec(int32_t level, int64_t p0, int64_t n, int32_t *out);

/* The chemistry's single-precision rate fits (Sec. 4.1: case-B and case-A
 * recombination, collisional ionisation of HI, and the cooling rate of
 * recombination, collisional ionisation and excitation and free-free
 * emission with unit electron, HI and HII densities, no Compton term) at n
 * temperatures T float[n] (K, 1 <= T <= 1e9): out float[4n] = (alpha_B,
 * alpha_A cm^3/s, C_HI cm^3/s, Lambda erg cm^3/s) per temperature.
 * FLEXRT_E_INVALID for a temperature out of range.  Synchronous. */
flexrt_status flexrt_probe_rates(int64_t n, const float *T, float *out);

/* Rotation of (seed, emitter, step) quantised to 2^24: out int32[9]. */
flexrt_status flexrt_probe_rotation(uint64_t seed, int64_t emitter, int64_t step,
                                    int32_t rotate, int32_t *out);

/* Rotated fixed-point directions of pixels p0..p0+n-1 at `level`:
 * round(Rq . vq / 2^27), out int32[3n]; Rq int32[9]. */
flexrt_status flexrt_probe_direction(int32_t level, int64_t p0, int64_t n,
                                     const int32_t *Rq, int32_t *out);

/* Merge-sphere pixel (Sec. 3.3) of n fixed-point directions d int32[3n] on
 * the sphere rotated by Rq at `level` (0..12): out int32[n].  Rq holds
 * n_rot rotations int32[9 * n_rot]: n_rot == 1, one sphere for every
 * direction; n_rot == n, direction i on sphere i.  The step's decision:
 * single precision, one fixed sequence of correctly rounded operations
 * (v = Rq^T d, NESTED ang2pix). */
flexrt_status flexrt_probe_merge_pixel(int32_t level, int64_t n, const int32_t *d, const int32_t *Rq,
                                       int64_t n_rot, int32_t *out);

/* Rays as the merge step sees them (flexrt_probe_merge): n rays, caller-owned
 * host arrays.  pixlev = level << 28 | NESTED pixel (merge pixel of a vertex
 * ray); emitter = emitter index, or 0x80000000 | local cell of the merge for
 * a merged ray; birth = birth step (merged: step of the merge); dir int32[3n]
 * (2^-21 cell per step); photons float[nbins * n] (code photons, bin
 * fastest); merged rays only: pos int32[3n] (position at the merge), aux =
 * vertex << 31 | distance travelled at the merge (cells), thr (termination
 * threshold, code photons). */
typedef struct {
    uint32_t *pixlev, *emitter;
    int32_t *birth, *dir;
    float *photons;
    int32_t *pos;
    uint32_t *aux;
    float *thr;
} flexrt_probe_rays;

/* One simulation's constants for flexrt_probe_merge: grid, bins, HEALPix
 * levels, K = floor(N_ex * N_RT), sphere seed and rotation switch, the step
 * whose march produced the rays, eps_term, and the emitters: cell int32[3*ne]
 * and this step's code photons per cast ray n0 float[ne]. */
typedef struct {
    int32_t nx, ny, nz, nbins;
    int32_t l_src, l_max, l_merge;
    int64_t k_ex;
    uint64_t seed;
    int32_t rotate, step;
    float eps_term;
    int32_t n_emitters;
    const int32_t *emitter_cell;
    const float *emitter_n0;
} flexrt_merge_probe;

/* The merge step (Sec. 3.3) alone: the very kernels of a step's merge run on
 * n host-given live rays (const in) of one simulation as they stand after the
 * march of step p->step.  Writes up to cap of the rays left live to out and
 * their number to *n_out, in the order the kernels leave them in the queue
 * (the rays that did not merge in their slots, then the merged rays, which
 * the merge appends; the slots of the rays that merged, empty, are
 * skipped).  Allocates and frees its own device scratch.  Synchronous. */
flexrt_status flexrt_probe_merge(const flexrt_merge_probe *p, int64_t n, const flexrt_probe_rays *in,
                                 int64_t cap, flexrt_probe_rays *out, int64_t *n_out);

/* One-step cell traversal (Sec. 3.1) of n rays from p0 (int64[3n], 2^-21
 * cell, |p0| < 2^31 - 2^22) along d (int32[3n], |d| <= 2^21) in grid g:
 * cells int32[n*4*3], ds float[n*4] (cells), nseg int32[n], escaped
 * int32[n].  FLEXRT_E_INVALID for coordinates out of range. */
flexrt_status flexrt_probe_traverse(int64_t n, const int64_t *p0, const int32_t *d,
                                    const flexrt_grid *g, int32_t *cells, float *ds,
                                    int32_t *nseg, int32_t *escaped);

/* ----------------------------------------------------------------------- */
/* Batch: many independent simulations of different sizes advanced by one  */
/* set of kernel launches per RT step (replayed from a CUDA graph).  Each   */
/* member follows exactly the single-simulation step above; the batch only  */
/* shares the launches, the ray queue and the device arenas.  Members can   */
/* be added and retired between steps (continuous batching).                */
/* ----------------------------------------------------------------------- */
typedef struct {
    int32_t max_sims;        /* simulation slots, 1..512                       */
    int32_t max_grid;        /* largest grid edge of any member                */
    int32_t nbins;           /* frequency bins of the ray layout (members may use fewer) */
    double n_ray_min;        /* N_min used to size the pixel table (members choose their own) */
    int64_t ray_capacity;    /* rays per queue, shared by all members; 0 = sized from free memory */
    int64_t cell_capacity;   /* cells of all members together                  */
    int32_t emitter_capacity;/* emitters of all members together               */
    int32_t keep_diagnostics;
    int32_t use_graph;       /* 1: replay each step from a CUDA graph          */
    void *cuda_stream;       /* 0 = library-owned stream                       */
    int32_t merge_l_max;     /* deepest l_merge members may use (its scratch is
                                cell_capacity * 12 * 4^merge_l_max groups);
                                -1: members cannot merge                       */
    int32_t gen_capable;     /* 1: members may run Generalized mode            */
    int64_t device_bytes_max;/* cap on the batch's device allocations (0 = none);
                                flexrt_batch_create fails with FLEXRT_E_OOM and
                                frees everything when the arenas exceed it     */
} flexrt_batch_config;

void flexrt_default_batch_config(flexrt_batch_config *c);

/* Allocates every device arena of the batch; later calls allocate nothing. */
flexrt_status flexrt_batch_create(const flexrt_batch_config *c, flexrt_batch **out);

/* Admit one simulation (same parameters as flexrt_create plus its sources and
 * step length): host inputs are copied before the call returns (the copies
 * to the device run in stream order, behind the steps already enqueued: the
 * call does not wait for them); *slot receives its slot.
 * FLEXRT_E_CAPACITY when no slot, cells or emitters are free. */
flexrt_status flexrt_batch_add(flexrt_batch *b, const flexrt_grid *grid, const flexrt_box *box,
                               const double *n_H, const flexrt_mfp *mfp, const flexrt_spectrum *spectrum,
                               const flexrt_options *opt, int32_t n_sources, const int32_t *cell_ijk,
                               const double *ndot, double dt_s, int32_t *slot);

/* Enqueue one RT step of every active member (asynchronous; errors latched
 * as for flexrt_step). */
flexrt_status flexrt_batch_step(flexrt_batch *b);
flexrt_status flexrt_batch_sync(flexrt_batch *b);

/* Remove a member between steps (without waiting for enqueued steps, which
 * still advance it); its cells are reusable at once, its slot and emitters
 * after the next step. */
flexrt_status flexrt_batch_retire(flexrt_batch *b, int32_t slot);

/* Per-member read-back, as the single-simulation getters. */
flexrt_status flexrt_batch_get_fields(flexrt_batch *b, int32_t slot, flexrt_fields *f);
flexrt_status flexrt_batch_get_budget(flexrt_batch *b, int32_t slot, double out[4]);
flexrt_status flexrt_batch_get_screen_excess(flexrt_batch *b, int32_t slot, double *photons);
flexrt_status flexrt_batch_get_counts(flexrt_batch *b, int32_t slot, int64_t out[6]);
flexrt_status flexrt_batch_get_segment_counts(flexrt_batch *b, int32_t slot, int32_t *out);
flexrt_status flexrt_batch_get_rays(flexrt_batch *b, int32_t slot, int64_t cap, int32_t *level,
                                    int64_t *pixel, int32_t *emitter, int32_t *birth, int32_t *dir,
                                    double *photons, int64_t *n);
flexrt_status flexrt_batch_get_ionized_volume(flexrt_batch *b, int32_t slot, double *x_ion);
flexrt_status flexrt_batch_get_rays_merged(flexrt_batch *b, int32_t slot, int64_t cap, int32_t *merged,
                                           int32_t *vertex, int32_t *dist, int64_t *pos, double *thr,
                                           int64_t *n);

/* out[0] active members, out[1] free cells, out[2] free emitters,
 * out[3] ray capacity, out[4] queue slots in use by live rays after the last
 * step seen complete (does not wait for enqueued steps; exact after
 * flexrt_batch_sync), out[5] free slots. */
flexrt_status flexrt_batch_info(flexrt_batch *b, int64_t out[6]);
flexrt_status flexrt_batch_set_launch(flexrt_batch *b, int32_t agg, int32_t minb, int32_t blocks_per_sm,
                                      int32_t threads, int32_t slab);
const char *flexrt_batch_last_error(const flexrt_batch *b);
void flexrt_batch_destroy(flexrt_batch *b);

/* Largest batch of flexrt_probe_traverse_static, in rays. */
#define FLEXRT_STATIC_MAX_RAYS 32768

/* flexrt_probe_traverse without any device allocation.  The paper has no
 * counterpart: this is a deployment facility.  It is for callers that must
 * not call cudaMalloc/cudaFree: programs whose device memory is owned by
 * another allocator that has reserved the device (a framework's caching
 * allocator, a fixed memory budget), and latency-sensitive loops that cannot
 * take the implicit device synchronisation of cudaFree.
 * Same arguments, results and kernel as flexrt_probe_traverse.  Its device
 * staging is one fixed array inside the library of about 3.5 MB
 * (FLEXRT_STATIC_MAX_RAYS rays), present on every GPU that loads the library
 * until the process exits.  n > FLEXRT_STATIC_MAX_RAYS returns
 * FLEXRT_E_CAPACITY with a message in flexrt_last_error(NULL).  The first call
 * on each device looks up the array's device address and keeps it for the
 * life of the process; make that first call before any stream capture.  A
 * device reset (cudaDeviceReset, or a reset of the primary context) between
 * calls is not supported: the kept address would be stale.  Every call reuses the same array: calls that
 * overlap on the GPU (e.g. from two host threads) race, so serialise them.
 * Synchronous; runs on the legacy default stream; allocates nothing. */
flexrt_status flexrt_probe_traverse_static(int64_t n, const int64_t *p0, const int32_t *d,
                                           const flexrt_grid *g, int32_t *cells, float *ds,
                                           int32_t *nseg, int32_t *escaped);

#ifdef __cplusplus
}
#endif
#endif
