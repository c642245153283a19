/*
 * mcrt.h -- C ABI of the GB300 null-collision Monte Carlo radiative-transfer
 * library (sm_103a).
 *
 * The library traces many independent photon paths through a voxelised
 * extinction field above a ground, sampling free paths by null collisions
 * over a pyramid of max-majorants, and scores radiance or ground-flux tallies
 * by local estimates toward the sun (Villefranque et al. 2019, "Path-tracing
 * Monte Carlo library for 3D radiative transfer in highly resolved cloudy
 * atmospheres"; Sec. 2.3, Eq. 2, Sec. 2.4, Sec. 3.1, Sec. 4.1).
 *
 * Conventions shared by every call
 *  - Units: km for lengths, km^-1 for extinction.  Axes x, y are periodic,
 *    z runs from the ground (z = 0) to the top of the field (z = nz * dz);
 *    above it the atmosphere is empty.
 *  - Arrays are row-major with x fastest: index ((z * ny) + y) * nx + x.
 *  - Handles are opaque and created/destroyed in pairs.  The library owns
 *    every device allocation it makes; caller buffers are borrowed for the
 *    duration of the call only and never freed by the library.
 *  - Every call returns an mcrt_status (0 = success, < 0 = error).  Nothing
 *    is thrown across the ABI and no device assert or trap is used; the text
 *    of the last error of a context is returned by mcrt_last_error().
 *  - Work is issued on the context's stream in call order.  Calls that
 *    return data to host memory synchronise that stream before returning.
 *  - Results depend only on the inputs and the seed, not on launch shape:
 *    path i draws its random numbers from Philox4x32-10 counters derived
 *    from (seed, i, event, stream).
 *  - A NULL handle or pointer where one is required gives MCRT_ERR_ARG.
 */
#ifndef MCRT_H
#define MCRT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MCRT_ABI_VERSION 2

#if defined(__GNUC__)
#define MCRT_API __attribute__((visibility("default")))
#else
#define MCRT_API
#endif

typedef struct mcrt_ctx mcrt_ctx;
typedef struct mcrt_scene mcrt_scene;
typedef struct mcrt_tally mcrt_tally;
typedef struct mcrt_proposal mcrt_proposal;

typedef enum {
    MCRT_OK = 0,
    MCRT_ERR_ARG = -1,        /* invalid argument (message says which)        */
    MCRT_ERR_OOM = -2,        /* device or host allocation failed             */
    MCRT_ERR_CUDA = -3,       /* a CUDA runtime call failed                   */
    MCRT_ERR_TIMEOUT = -4,    /* the trace deadline expired; tallies partial  */
    MCRT_ERR_CANCELLED = -5,  /* the cancel flag was raised; tallies partial  */
    MCRT_ERR_STATE = -6,      /* call out of order (e.g. no majorants yet)    */
    MCRT_ERR_BOUNDS = -7,     /* an output buffer is too small                */
    MCRT_ERR_UNSUPPORTED = -8 /* valid request the library does not handle    */
} mcrt_status;

enum { MCRT_MEM_HOST = 0, MCRT_MEM_DEVICE = 1 };
enum { MCRT_STORAGE_F32 = 0, MCRT_STORAGE_BF16 = 1 };
/* Sun transmissivity estimators: ratio tracking (Sec. 2.3's null-collision
 * algorithm scoring 1 - k/M per tentative collision), delta tracking (its
 * 0/1 form), decomposition tracking (each leaf's minorant m is a control
 * whose exp(-m s) is applied exactly; ratio tracking on k - m with majorant
 * M - m; a voxel leaf is crossed without random draws). */
enum { MCRT_SUN_RATIO = 0, MCRT_SUN_DELTA = 1, MCRT_SUN_DECOMP = 2 };

/* Phase function of the clear-air part of the field (Sec. 4.1: gas
 * molecules scatter by Rayleigh, droplets by Henyey-Greenstein). */
enum { MCRT_PHASE_HG = 0, MCRT_PHASE_RAYLEIGH = 1 };

/* Max grid a trace tracks through (mcrt_trace_opts.grid): the 8^L pyramid
 * (level-L cells of 8^L voxels per axis), or the paper's octree (Sec.
 * 3.1.1: groups of 2^3 cells merged recursively, level-L cells of 2^L
 * voxels per axis), which mcrt_scene_build_octree must have built. */
enum { MCRT_GRID_PYRAMID = 0, MCRT_GRID_OCTREE = 1 };

/* Order in which a camera trace claims its pixels (mcrt_trace_opts.pixel_order). */
enum { MCRT_ORDER_COST = 0, MCRT_ORDER_RASTER = 1 };

/* How a camera trace schedules its paths on the GPU (mcrt_trace_opts.schedule).
 * PERSISTENT: one loop per GPU thread that takes one step of one path per
 * iteration, path state in registers (the default).  WAVEFRONT: paths wait
 * in structure-of-arrays queues in device memory between stages (flight
 * tracking; vertex and sun ray; path start), one kernel per stage and round.
 * Both compute the same path scores bit for bit (Philox counters and FP32
 * steps are the same); only the order of the FP64 tally additions differs.
 * The wavefront form serves plain camera images only: no proposal, shards,
 * decomposition tracking, Rayleigh clear air, heightfield ground, event
 * counts, deadline or cancel flag (MCRT_ERR_UNSUPPORTED), and not through
 * mcrt_trace_flux, mcrt_trace_batch or the no-allocation call. */
enum { MCRT_SCHEDULE_PERSISTENT = 0, MCRT_SCHEDULE_WAVEFRONT = 1 };

/* Library version and the ABI version it was built with. */
MCRT_API int mcrt_version(int32_t* abi_version);

/* Text for a status code (static storage, never NULL). */
MCRT_API const char* mcrt_status_string(int status);

/* --------------------------------------------------------------------- */
/* Context                                                                */
/* --------------------------------------------------------------------- */

/* Create a context on CUDA device `device`.  `cuda_stream` is a
 * cudaStream_t borrowed from the caller (it may be a framework's current
 * stream) or NULL for the legacy default stream; it must outlive the
 * context.  Errors: MCRT_ERR_ARG (bad device or NULL out), MCRT_ERR_CUDA. */
MCRT_API int mcrt_create(mcrt_ctx** out, int device, void* cuda_stream);

/* Destroy a context after its scenes and tallies.  Synchronises its stream. */
MCRT_API int mcrt_destroy(mcrt_ctx* ctx);

/* Last error message of the context ("" if none); valid until the next call
 * on the context. */
MCRT_API const char* mcrt_last_error(const mcrt_ctx* ctx);

/* Number of kernels this context has launched so far (all calls). */
MCRT_API int mcrt_launch_count(const mcrt_ctx* ctx, uint64_t* count);

/* --------------------------------------------------------------------- */
/* Scene: the extinction field, its majorant pyramid, ground and sun.     */
/* --------------------------------------------------------------------- */

typedef struct {
    int32_t nx, ny, nz;        /* voxels per axis, each >= 1                   */
    float dx, dy, dz;          /* voxel size [km], > 0                          */
    const float* ext;          /* total extinction k [km^-1], nx*ny*nz values,  */
                               /* finite and >= 0, x fastest                    */
    int32_t ext_mem;           /* MCRT_MEM_HOST or MCRT_MEM_DEVICE              */
    float k_clear;             /* uniform clear-sky part of k [km^-1]           */
    float ssa_clear;           /* single-scattering albedo of the clear part    */
    float ssa_cloud;           /* single-scattering albedo of k - k_clear       */
    float hg_g;                /* Henyey-Greenstein asymmetry, |g| < 1          */
    int32_t storage;           /* MCRT_STORAGE_F32, or MCRT_STORAGE_BF16:       */
                               /* voxels rounded to nearest bf16, majorants     */
                               /* rounded up so they stay bounds               */
} mcrt_field_desc;

/* Create a scene from a field description.  The field is copied (from host
 * or device memory) into the library's brick-major layout: 8x8x8 voxel
 * bricks, 2 KiB each (Sec. 3.1.2: fixed-size blocks of spatially coherent
 * voxels).  Single-scattering albedo at a voxel is
 *   omega = ((k - k_clear) * ssa_cloud + k_clear * ssa_clear) / k
 * (cloud droplets and clear air mixed in proportion to their extinction,
 * Sec. 4.1 species sampling in expectation).  The ground is black and the
 * sun at zenith until set.  A host field in page-locked memory mapped
 * into the device's address space (cudaHostAlloc, or cudaHostRegister with
 * cudaHostRegisterMapped) is read by the relayout kernel directly; other
 * host memory is copied to a device staging buffer first.  Errors:
 * MCRT_ERR_ARG, MCRT_ERR_OOM, MCRT_ERR_CUDA. */
MCRT_API int mcrt_scene_create(mcrt_ctx* ctx, const mcrt_field_desc* desc, mcrt_scene** out);

/* Destroy a scene (synchronises the context stream). */
MCRT_API int mcrt_scene_destroy(mcrt_scene* scene);

/* Build the majorant pyramid: level 0 is the voxel field, a level-L cell
 * covers 8^L voxels per axis (clipped at the field edges) and holds the
 * exact max of its children (Sec. 3.1.1: merged voxels keep the max
 * extinction; Sec. 2.4: the majorant is uniform by parts).  `levels` >= 1
 * levels are built above the voxels; 0 builds up to the first level with
 * one cell.  Errors: MCRT_ERR_ARG (levels < 0 or > 8). */
MCRT_API int mcrt_scene_build_majorants(mcrt_scene* scene, int32_t levels);

/* Number of majorant levels built (0 if none). */
MCRT_API int mcrt_scene_levels(const mcrt_scene* scene, int32_t* levels);

/* Cells per axis of level `level` (1..levels). */
MCRT_API int mcrt_scene_majorant_dims(const mcrt_scene* scene, int32_t level, int32_t dims[3]);

/* Copy level `level` of the pyramid (x fastest) into host memory.
 * `n` must be at least the level's cell count (else MCRT_ERR_BOUNDS);
 * MCRT_ERR_STATE before mcrt_scene_build_majorants. */
MCRT_API int mcrt_scene_read_majorants(const mcrt_scene* scene, int32_t level, float* host_out, size_t n);

/* The minorant pyramid built with the majorants (exact min over each
 * cell's existing children; for BF16 storage, the min of the stored
 * values), read like mcrt_scene_read_majorants.  It is the control of
 * decomposition tracking (MCRT_SUN_DECOMP); the paper's octree keeps the
 * min beside the max (Sec. 3.1.1). */
MCRT_API int mcrt_scene_read_minorants(const mcrt_scene* scene, int32_t level, float* host_out, size_t n);

/* Build the paper's octree (Sec. 3.1.1) beside the pyramid: a level-L cell
 * covers an aligned block of 2^L voxels per axis (clipped at the field
 * edges) and holds the max and the min of the voxels it covers, as stored
 * (for BF16 storage the nearest-bfloat16 values, so the max bounds exactly
 * what the tracer reads).  `levels` >= 1 levels are built; 0 builds up to
 * the first level with one cell.  Traces choose it with
 * mcrt_trace_opts.grid = MCRT_GRID_OCTREE; its leaves follow the same
 * tau~ rule with h_z = dz 2^L.  Device memory: about 8/7 x (cells of level
 * 1) x 16 bytes (max, min and the leaf map).  Rebuilding replaces it.
 * Errors: MCRT_ERR_ARG (levels < 0 or > 20), MCRT_ERR_OOM, MCRT_ERR_CUDA. */
MCRT_API int mcrt_scene_build_octree(mcrt_scene* scene, int32_t levels);

/* Octree levels built (0 if none), and the cells per axis of one level. */
MCRT_API int mcrt_scene_octree_levels(const mcrt_scene* scene, int32_t* levels);
MCRT_API int mcrt_scene_octree_dims(const mcrt_scene* scene, int32_t level, int32_t dims[3]);

/* Copy level `level` (1..levels) of the octree, x fastest, into host
 * memory: maxima into max_out and minima into min_out (either may be
 * NULL).  `n` must be at least the level's cell count (else
 * MCRT_ERR_BOUNDS); MCRT_ERR_STATE before mcrt_scene_build_octree. */
MCRT_API int mcrt_scene_read_octree(const mcrt_scene* scene, int32_t level, float* max_out, float* min_out, size_t n);

/* Flat Lambertian ground of albedo in [0, 1] (Sec. 4.1). */
MCRT_API int mcrt_scene_set_ground_flat(mcrt_scene* scene, float albedo);

/* Phase function of the clear air (k_clear, omega_clear): MCRT_PHASE_HG
 * (default: the droplets' g) or MCRT_PHASE_RAYLEIGH, 3 (1 + mu^2) / (16 pi).
 * With Rayleigh, a scattering vertex uses the mixture of the two species'
 * phase functions weighted by their scattering coefficients in its local
 * estimate, and samples the species (Sec. 4.1) before its direction.  Not
 * available with a learned proposal or in batches. */
MCRT_API int mcrt_scene_set_clear_sky_phase(mcrt_scene* scene, int32_t phase);

/* Heightfield ground instead of the flat one (an extension of the paper's
 * flat Lambertian ground, Sec. 1 and Sec. 4.1).  heights: hny rows of hnx
 * FP32 heights [km] (x fastest) at the corners of a periodic grid of
 * hnx x hny cells spanning the field's x-y extent; each cell is cut along
 * the diagonal from corner (i, j) to (i+1, j+1) into two planar triangles.
 * mem: MCRT_MEM_HOST or MCRT_MEM_DEVICE (borrowed for the call, copied).
 * Heights must be finite and in [0, nz * dz] (MCRT_ERR_ARG otherwise).
 * Paths end their flights on the surface, sun rays that meet it are
 * shadowed, ground vertices use the facet normal (Lambertian about it,
 * local estimate rho/pi * max(n.s, 0) * T_sun), and the flux sensor sits
 * on the surface: per unit horizontal area, T_dir = max(n.s, 0) / (n_z mu0)
 * * T_sun and T_dif = pi / (n_z mu0) * sum of estimates.  A max pyramid of
 * 4 x 4 blocks (while both sizes divide) lets rays skip terrain below them.
 * Not available with a learned proposal or in batches. */
MCRT_API int mcrt_scene_set_ground_heightfield(mcrt_scene* scene, const float* heights, int32_t hnx, int32_t hny,
                                               int32_t mem, float albedo);

/* Collimated sun; zenith in [0, 90) degrees, azimuth measured from +x
 * toward +y (App. C scene table convention).  Direction toward the sun:
 * (sin z cos a, sin z sin a, cos z). */
MCRT_API int mcrt_scene_set_sun(mcrt_scene* scene, float zenith_deg, float azimuth_deg);

/* --------------------------------------------------------------------- */
/* Tracing                                                                */
/* --------------------------------------------------------------------- */

/* Pinhole camera (Sec. 4.1, App. C table of camera set-ups): position,
 * target point, up vector, horizontal field of view and image size.  Pixel
 * (px, py) spans image-plane coordinates
 *   sx = (2 (px + jx) / width - 1) tan(fov / 2),
 *   sy = (2 (py + jy) / height - 1) tan(fov / 2) height / width,
 * jx, jy uniform jitter; direction = normalise(f + sx r + sy u) with
 * f = normalise(target - pos), r = normalise(f x up), u = r x f.
 * Image rows are py, columns px. */
typedef struct {
    float pos[3];
    float target[3];
    float up[3];
    float fov_deg;
    int32_t width, height;
} mcrt_camera_desc;

typedef struct {
    float tau_merge;           /* leaf threshold tau~ (Sec. 4.2): a cell of     */
                               /* level > finest_level is tracked whole when   */
                               /* its majorant times its height is <= tau~;    */
                               /* INFINITY = coarsest level.  Default 1.        */
    int32_t finest_level;      /* finest level tracked: 0 (default: a voxel is  */
                               /* its own leaf where no coarser cell qualifies, */
                               /* as unmerged voxels in Sec. 4.2), or 1 (level- */
                               /* 1 cells are always merged)                    */
    int32_t max_order;         /* 0: all scattering orders; n: score events of  */
                               /* order <= n and stop after order n             */
    int32_t sun_mode;          /* MCRT_SUN_RATIO (default), _DELTA or _DECOMP   */
    int32_t chunk;             /* paths a GPU thread claims at once; 0 = auto:  */
                               /* 1, 2, 4 or 8 as the paths per                 */
                               /* resident thread pass 48, 160 and 400 (camera: */
                               /* dividing spp; batch: 4).  Launch shape only   */
    int32_t block_size;        /* threads per block; 0 = auto                   */
    int32_t grid_size;         /* blocks; 0 = SMs x resident blocks             */
    int32_t count_events;      /* 1: also count collisions and leaf steps       */
    int32_t rare_batch;        /* GPU lanes of a warp that must be waiting for  */
                               /* a path start, ray start or vertex before that */
                               /* work runs (1..32; 0 = default 10).  Launch    */
                               /* shape only: results do not depend on it       */
    struct mcrt_proposal* proposal; /* NULL: plain HG sampling.  Else the first */
                               /* n_learned volume vertices of every path draw  */
                               /* their direction by one-sample MIS from        */
                               /* alpha p_HG + (1 - alpha) q_network, weight    */
                               /* p_HG / q (unbiased for any network)           */
    int32_t n_learned;         /* 0 = 8                                         */
    float mis_alpha;           /* HG share alpha in (0, 1]; 0 = 0.5             */
    int32_t learn;             /* 1: after each batch of paths, train the       */
                               /* network (Adam) on the vertices that batch     */
                               /* produced; the first batch of an untrained     */
                               /* network samples HG only                       */
    int32_t batch_paths;       /* paths per batch in learned mode; 0 = 2^21     */
                               /* when learning, else 2^25 (about 12 GB of      */
                               /* queues; larger batches waste less time in     */
                               /* the passes' tails)                            */
    float learning_rate;       /* 0 = 1e-3                                      */
    int32_t train_steps;       /* Adam steps per batch; 0 = 1                   */
    double deadline_ms;        /* > 0: stop and report MCRT_ERR_TIMEOUT after   */
                               /* this much device time                         */
    const volatile int32_t* cancel_flag; /* NULL, or a flag in host-mapped or   */
                               /* device memory; non-zero stops the trace with  */
                               /* MCRT_ERR_CANCELLED                            */
    int32_t batch_dalpha;      /* batches: 1 also estimates dT/dalpha (the 5th   */
                               /* quantity; 0 leaves it 0 and runs faster)      */
    int32_t grid;              /* MCRT_GRID_PYRAMID (default) or                */
                               /* MCRT_GRID_OCTREE: the max grid tracked        */
    int32_t pixel_order;       /* camera traces: MCRT_ORDER_COST (default)      */
                               /* claims the pixels whose view ray crosses the  */
                               /* most majorant optical depth first (a short    */
                               /* pre-pass per 8x8 tile), so the longest paths  */
                               /* do not start last; MCRT_ORDER_RASTER claims   */
                               /* them row by row.  Launch shape only: a path's */
                               /* id, draws and result do not depend on it      */
    int32_t shard_index;       /* shard_count > 1: trace one shard of the paths */
    int32_t shard_count;       /* (one process per GPU, Sec. 3's independent    */
                               /* paths).  Camera: the pixels at positions      */
                               /* shard_index, + shard_count, ... of the claim  */
                               /* order (pixel_order), all spp paths of each;   */
                               /* flux: path ids [n*i/c, n*(i+1)/c).  Paths keep */
                               /* their global ids, so the shards' FP64 sums    */
                               /* (mcrt_tally_read_sums) add up to the whole    */
                               /* trace's; a shard's own mean divides by the   */
                               /* whole path count.  0 or 1: no sharding.  Not  */
                               /* with a proposal, in batches or without        */
                               /* allocation (MCRT_ERR_UNSUPPORTED)             */
    int32_t schedule;          /* MCRT_SCHEDULE_PERSISTENT (default) or         */
                               /* MCRT_SCHEDULE_WAVEFRONT (camera traces)       */
    int32_t wavefront_slots;   /* wavefront: paths in flight (queue entries per */
                               /* stage, 80 B each, three queues); 0 = 2^21,    */
                               /* at most 2^26.  Launch shape only              */
} mcrt_trace_opts;

/* Fill `opts` with the defaults listed above. */
MCRT_API int mcrt_trace_opts_default(mcrt_trace_opts* opts);

/* Backward radiance image (Sec. 4.1): for each pixel, `spp` paths start at
 * the camera; path p of pixel q has global id q * spp + p.  At every volume
 * collision x the path scores  w * omega(x) * p_HG(d . s) * T_sun(x)  and at
 * every ground hit  w * (albedo / pi) * max(s_z, 0) * T_sun(x), where w is
 * the product of albedos met so far, d the path direction and s the sun
 * direction; T_sun is estimated by ratio (or delta) tracking through the
 * same majorants (Sec. 2.3).  Directions are resampled from HG or the
 * cosine law; Russian roulette below w = 0.01.  Radiance is in units of the
 * solar irradiance per sr.  The tally has width*height cells, 1 quantity.
 * *tally_inout: NULL to create a new tally, or an existing tally of the same
 * shape to reuse (its sums are reset).  Requires majorants.  The paths run
 * in one persistent kernel, or with opts->schedule = MCRT_SCHEDULE_WAVEFRONT
 * as stage kernels over device queues (same path scores).  Errors:
 * MCRT_ERR_ARG, MCRT_ERR_STATE, MCRT_ERR_TIMEOUT, MCRT_ERR_CANCELLED,
 * MCRT_ERR_UNSUPPORTED, MCRT_ERR_CUDA, MCRT_ERR_OOM. */
MCRT_API int mcrt_trace_camera(mcrt_scene* scene, const mcrt_camera_desc* camera, uint32_t spp, uint64_t seed,
                      const mcrt_trace_opts* opts, mcrt_tally** tally_inout);

/* Domain-mean ground transmittance (Sec. 5.1, 5.2): `npaths` paths start at
 * uniform ground points with cosine-distributed upward directions.  The tally
 * has 1 cell and 3 quantities: T_dir = sun transmissivity from the ground
 * point, T_dif = (pi / mu0) * sum of local estimates, T_tot = T_dir + T_dif;
 * all normalised by mu0 times the solar irradiance. */
MCRT_API int mcrt_trace_flux(mcrt_scene* scene, uint64_t npaths, uint64_t seed, const mcrt_trace_opts* opts,
                    mcrt_tally** tally_inout);

/* Camera trace that allocates no device memory (the paper has no
 * counterpart; this is a convenience for callers that cannot allocate GPU
 * memory while tracing -- code living inside another framework's memory
 * budget, real-time loops that must not touch the allocator).  Same physics,
 * random numbers and options as mcrt_trace_camera, but the working memory
 * (work counter, status, FP64 per-pixel sums) is one statically sized
 * device array inside the library, and the per-pixel mean and standard
 * error (row-major, width * height doubles each) are written to d_mean and
 * d_stderr, device buffers owned by the caller.
 *  - At most 65536 pixels (256 x 256); larger images return
 *    MCRT_ERR_BOUNDS before any GPU work.
 *  - The array (about 1 MiB) stays allocated on every GPU that loads the
 *    library until the process exits.
 *  - All calls share it: each call clears what it uses first, but calls
 *    whose GPU work overlaps (several streams or threads on one device)
 *    race.  Issue them one after another on one stream.
 *  - The first call on a device looks up the array's device address; make
 *    that first call before capturing any stream.
 *  - Pixels are claimed in raster order whatever opts->pixel_order says (the
 *    cost order needs work buffers); results are the same either way.
 *  - The scene's majorants must be built.  Synchronises the context stream;
 *    errors as mcrt_trace_camera plus MCRT_ERR_BOUNDS, and
 *    MCRT_ERR_UNSUPPORTED for a learned proposal or a shard (they need work
 *    buffers).  After MCRT_ERR_TIMEOUT or MCRT_ERR_CANCELLED both output
 *    buffers hold NaN (the partial sums estimate nothing). */
MCRT_API int mcrt_trace_camera_noalloc(mcrt_scene* scene, const mcrt_camera_desc* camera, uint32_t spp, uint64_t seed,
                                       const mcrt_trace_opts* opts, double* d_mean, double* d_stderr);

/* Many flux problems in one persistent launch (paths of all items share one
 * work queue; the paper builds one grid per spectral quadrature point and
 * traces them separately, Sec. 3.1.1 and Sec. 6).  Item i traces npaths
 * ground-flux paths through its scene with an extra uniform pure absorber
 * k_gas (a spectral band's gas: majorants become M + k_gas, so one pyramid
 * serves every band) under its own sun; path j of an item draws exactly the
 * random numbers path j of mcrt_trace_flux with the item's seed draws.  The
 * tally has n cells x 5 quantities: T_dir, T_dif, T_tot, dT_tot/dg (the
 * derivative with respect to the HG asymmetry, by the score-function
 * method) and dT_tot/dalpha (with respect to the cloud droplets'
 * absorptivity alpha = 1 - omega_cloud at fixed extinction, the sensitivity
 * of Sec. 6.1: each estimate times the sum of d ln omega / d alpha over the
 * path's volume vertices so far; only with opts->batch_dalpha, else 0),
 * both along the same paths.  Scenes must have majorants; items must
 * share FP32 or BF16 storage.  The learned proposal is not used here. */
typedef struct {
    const mcrt_scene* scene;
    float k_gas;               /* gas absorption of the band [km^-1], >= 0     */
    float sun_zenith_deg;      /* [0, 90)                                       */
    float sun_azimuth_deg;
    uint64_t npaths;           /* >= 1                                          */
    uint64_t seed;
} mcrt_batch_item;

MCRT_API int mcrt_trace_batch(mcrt_ctx* ctx, const mcrt_batch_item* items, int32_t n, const mcrt_trace_opts* opts,
                              mcrt_tally** tally_inout);

/* Launch-shape autotuner for a batch: times mcrt_trace_batch on a fraction
 * of every item's paths for each candidate (paths per claim 1, 2, 4, 8;
 * rare-phase wait 4, 8, 12 lanes; 64 or 128 threads per block; the better
 * of two runs each) and writes the fastest into *opts_inout (*best_ms: its
 * time).  Too small a fraction lets the last, straggling paths dominate;
 * a quarter of the paths or more tunes for the full batch.  Results of a trace do
 * not depend on these choices, only its speed. */
MCRT_API int mcrt_autotune_batch(mcrt_ctx* ctx, const mcrt_batch_item* items, int32_t n, double path_fraction,
                                 mcrt_trace_opts* opts_inout, float* best_ms);

/* A batch prepared once and replayed: the items are laid out on the device
 * and the whole batch (tally reset, the persistent trace kernel, finalize,
 * copies of the results and the status to pinned host memory) is captured
 * into one CUDA graph, so a run costs one graph launch.  The scenes must
 * outlive the plan and keep their majorants; a run traces the same paths
 * again unless mcrt_batch_plan_set_seeds changes the seeds.  A run checks
 * its scenes first: if one changed since the plan was made (a trace with
 * another tau~, finest level or grid rebuilt its leaf map, its octree or
 * pyramid was rebuilt, its ground or phase function was set), the plan's
 * leaf maps are rebuilt and its item records remade before the launch.  Deadline and
 * cancel flag are not available in plans (MCRT_ERR_UNSUPPORTED).
 * mcrt_batch_plan_run: mean and se (either may be NULL) receive n x 5
 * entries in the order of mcrt_trace_batch; *kernel_ms the graph's device
 * time (the trace kernel plus microseconds of reset, finalize and copies).  mcrt_batch_plan_tally lends the plan's tally (owned by the plan;
 * do not destroy it) for mcrt_tally_read and friends. */
typedef struct mcrt_batch_plan mcrt_batch_plan;

MCRT_API int mcrt_batch_plan_create(mcrt_ctx* ctx, const mcrt_batch_item* items, int32_t n,
                                    const mcrt_trace_opts* opts, mcrt_batch_plan** out);
MCRT_API int mcrt_batch_plan_set_seeds(mcrt_batch_plan* plan, const uint64_t* seeds, int32_t n);
MCRT_API int mcrt_batch_plan_run(mcrt_batch_plan* plan, double* mean, double* se, size_t count, float* kernel_ms);
MCRT_API int mcrt_batch_plan_tally(const mcrt_batch_plan* plan, const mcrt_tally** tally);
MCRT_API int mcrt_batch_plan_destroy(mcrt_batch_plan* plan);

/* --------------------------------------------------------------------- */
/* Tallies                                                                */
/* --------------------------------------------------------------------- */

/* Cells and quantities of a tally. */
MCRT_API int mcrt_tally_shape(const mcrt_tally* tally, int32_t* ncells, int32_t* nquant);

/* Mean, standard error of the mean and path count per (cell, quantity), cell
 * major; computed on the device from FP64 sums s1 = sum x, s2 = sum x^2:
 * mean = s1 / N, se = sqrt((s2 / N - mean^2) / (N - 1)).  Any output may be
 * NULL.  `count` must be >= ncells * nquant (else MCRT_ERR_BOUNDS). */
MCRT_API int mcrt_tally_read(const mcrt_tally* tally, double* mean, double* stderr_out, uint64_t* n, size_t count);

/* Raw FP64 sums (s1, s2) per (cell, quantity). */
MCRT_API int mcrt_tally_read_sums(const mcrt_tally* tally, double* s1, double* s2, size_t count);

/* Event counters of the trace that filled the tally (zeros unless
 * count_events was set): [0] paths, [1] tentative collisions on paths,
 * [2] real collisions, [3] ground hits, [4] leaf steps on paths,
 * [5] tentative collisions on sun rays, [6] leaf steps on sun rays,
 * [7] sun rays, [8] aborted paths (step guard), [9] free flights started,
 * and, when n >= 13: [10] most loop iterations spent on one path, [11] the
 * longest time in ns a GPU warp ran before the work queue ran dry, [12] the
 * longest time in ns a warp ran in total, and when n >= 22, [13..21] SM
 * clock cycles summed over warps spent in the sections of the trace loop
 * (loop top, random block, path start, ray start, step, vertex, load,
 * after-load, ray/path end), and when n >= 30, [22..29] lane occupancy
 * summed over warp iterations: iterations, lanes holding a path, lanes
 * taking a traversal step, of those at a tentative collision, lanes running
 * a batched rare phase (path start, ray start, vertex), lanes waiting for
 * one, iterations that ran rare phases, lanes with no path.  n >= 10. */
MCRT_API int mcrt_tally_counters(const mcrt_tally* tally, uint64_t* counters, size_t n);

/* Device time of the trace kernel that filled the tally, in ms. */
MCRT_API int mcrt_tally_kernel_ms(const mcrt_tally* tally, float* ms);

MCRT_API int mcrt_tally_destroy(mcrt_tally* tally);

/* --------------------------------------------------------------------- */
/* Learned scattering proposal (a project addition; the paper has none).  */
/* A 9-64-64-64-40 network (GELU, tanh form) maps the features of a volume */
/* vertex -- position scaled to [-1, 1] per axis, incoming direction, and  */
/* ln(k + 1e-6), ln(M1 + 1e-6), ln(M2 + 1e-6) of the voxel and its level-1 */
/* and level-2 majorants -- to an 8-lobe von Mises-Fisher mixture (per     */
/* lobe: axis, concentration softplus(.) + 1e-3, softmax weight).  The     */
/* tracer draws the new direction by one-sample MIS from                  */
/* q = alpha p_HG + (1 - alpha) q_vMF and multiplies the path weight by   */
/* p_HG / q, so the estimate stays unbiased for any network.              */
/* Parameters: 11,560 floats in the order W1[64][9], b1[64], W2[64][64],  */
/* b2[64], W3[64][64], b3[64], W4[40][64], b4[40] (row = output unit).    */
/* Inference and training run on the tensor cores in BF16 with FP32      */
/* accumulation; training keeps FP32 master weights and Adam moments.     */
/* --------------------------------------------------------------------- */
/* Number of network parameters (11,560). */
MCRT_API int mcrt_proposal_nparams(int32_t* n);

/* New network with Xavier-uniform weights drawn from Philox(seed) and zero
 * biases; Adam state cleared. */
MCRT_API int mcrt_proposal_create(mcrt_ctx* ctx, uint64_t seed, mcrt_proposal** out);
MCRT_API int mcrt_proposal_destroy(mcrt_proposal* proposal);

/* Copy parameters in from / out to host memory (n = 11,560).  Setting
 * clears the Adam state. */
MCRT_API int mcrt_proposal_set_params(mcrt_proposal* proposal, const float* host, size_t n);
MCRT_API int mcrt_proposal_get_params(const mcrt_proposal* proposal, float* host, size_t n);

/* The Adam state (first and second moments, n = 11,560 each, and the step
 * count) out to / in from host memory, for checkpoints: a network restored
 * with mcrt_proposal_set_params and then this call continues training
 * exactly where it stopped.  Set after the parameters (setting those clears
 * the state).  Errors: MCRT_ERR_BOUNDS (n too small), MCRT_ERR_ARG (a
 * moment not finite, a negative second moment, a bad step count). */
MCRT_API int mcrt_proposal_get_adam(const mcrt_proposal* proposal, float* host_m, float* host_v, size_t n,
                                    int64_t* step);
MCRT_API int mcrt_proposal_set_adam(mcrt_proposal* proposal, const float* host_m, const float* host_v, size_t n,
                                    int64_t step);

/* Evaluate the network on n feature rows (host, n x 9 floats, rounded to
 * BF16 on the device as in the tracer).  host_mix receives n x 40 mixture
 * parameters (per lobe: unit axis (3), concentration, weight); host_raw, if
 * not NULL, the n x 40 raw outputs. */
MCRT_API int mcrt_proposal_eval(mcrt_proposal* proposal, const float* host_features, size_t n, float* host_mix,
                                float* host_raw);

/* One training step on n records (host): features (n x 9), sampled
 * directions (n x 3) and target weights (n).  The loss is the mean of
 * -t log q_vMF(direction); the gradient of that mean is written to
 * host_grad (11,560, may be NULL) and, when lr > 0, one Adam step
 * (beta 0.9, 0.999, eps 1e-8) is applied.  *loss_out gets the loss. */
MCRT_API int mcrt_proposal_train_step(mcrt_proposal* proposal, const float* host_features, const float* host_dirs,
                                      const float* host_targets, size_t n, float lr, float* loss_out, float* host_grad);

/* One Adam step (beta 0.9, 0.999, eps 1e-8, learning rate lr > 0) with a
 * gradient the caller supplies (host, 11,560 floats, all finite): with
 * several processes, each computes its gradient with
 * mcrt_proposal_train_step(lr = 0), the processes average them, and each
 * applies the same average here, so every copy of the network stays the
 * same (data-parallel training).  Errors: MCRT_ERR_ARG. */
MCRT_API int mcrt_proposal_apply_gradient(mcrt_proposal* proposal, const float* host_grad, float lr);

/* Gradient kernel used by training steps (here and in traces that learn):
 * MCRT_TRAIN_TENSOR (default) runs every dense product of the forward and
 * backward passes on the tensor cores (BF16 operands, FP32 accumulation);
 * MCRT_TRAIN_FP32 runs them in FP32 on the CUDA cores.  Master weights and
 * Adam moments are FP32 either way. */
enum { MCRT_TRAIN_TENSOR = 0, MCRT_TRAIN_FP32 = 1 };
MCRT_API int mcrt_proposal_set_training(mcrt_proposal* proposal, int32_t mode);

/* --------------------------------------------------------------------- */
/* Checks (used by the tests; not on the hot path)                        */
/* --------------------------------------------------------------------- */

/* Leaves crossed by one ray, computed on the device with the tracer's own
 * traversal code: for each leaf (level, ix, iy, iz) in `cells` (4 int32 each)
 * and (t_in, t_out) in `t_in_out` (2 floats each, distances from o).
 * *status: 1 top reached, 2 ground reached, 3 capacity reached, 4 step
 * guard.  Host buffers.  Requires majorants. */
MCRT_API int mcrt_debug_dda(const mcrt_scene* scene, const float o[3], const float d[3], float tau_merge,
                   int32_t finest_level, int32_t* cells, float* t_in_out, int32_t cap, int32_t* count,
                   int32_t* status);

/* The same over a chosen grid (MCRT_GRID_PYRAMID or MCRT_GRID_OCTREE); a
 * leaf's (level, ix, iy, iz) are then that grid's level and cell index. */
MCRT_API int mcrt_debug_dda_grid(const mcrt_scene* scene, const float o[3], const float d[3], float tau_merge,
                                 int32_t finest_level, int32_t grid, int32_t* cells, float* t_in_out, int32_t cap,
                                 int32_t* count, int32_t* status);

/* Heightfield checks (MCRT_ERR_STATE on a flat ground): t_out[i] = the
 * distance t along ray i, o + t d (host arrays of n x 3 floats), to its
 * first surface hit, or +inf; and the surface height and unit normal at
 * n points (xy: n x 2; zn_out: n x 4 = z, nx, ny, nz). */
MCRT_API int mcrt_debug_terrain(const mcrt_scene* scene, int32_t n, const float* o, const float* d, float* t_out);
MCRT_API int mcrt_debug_terrain_height(const mcrt_scene* scene, int32_t n, const float* xy, float* zn_out);

/* Bounds-checked build (built with -DMCRT_CHECKED): *checked_build = 1 and
 * *count = the index violations the trace kernels have recorded since the
 * last call (then cleared), *first_code the first one's kind (1 voxel,
 * 2 leaf-map entry, 3 tally entry, 4 heightfield corner, 5 heightfield
 * pyramid cell); such an index is clamped, never followed.  In the normal
 * build *checked_build = 0 and *count = 0.  Synchronises the context
 * stream. */
MCRT_API int mcrt_debug_bounds_violations(mcrt_ctx* ctx, int32_t* checked_build, uint64_t* count,
                                          int32_t* first_code);

/* Device memory held by the allocations of the context's device's current
 * stream-ordered memory pool (the pool every allocation of this library
 * draws from, except a batch plan's item table): *used_current now and
 * *used_high the most since the last reset; reset_high != 0 then resets the
 * high mark to the current use.  Lets a caller check that a call allocated
 * nothing (the paper has no counterpart).  Synchronises the context
 * stream. */
/* The online-training records of one learned trace, for checks against an
 * independent implementation: the trace runs as mcrt_trace_camera
 * (camera != NULL, n = samples per pixel) or mcrt_trace_flux (n paths) with
 * opts->proposal and opts' n_learned and mis_alpha, in one batch of at most
 * 2^24 paths, without training the network.  Every learned vertex of a
 * path (one-sample MIS, the project's addition to the method of Sec. 4.1)
 * yields a record; the first min(cap, *count) are written in the order the
 * vertices were reached within each pass: feat (cap x 9) the vertex
 * features as the network saw them (BF16 values), dir (cap x 3) the sampled
 * direction, val (cap x 4) the path's score before the vertex, w * omega,
 * the vertex's own local estimate, and the target of the KL estimator
 * (score after the vertex without its own estimate, over w * omega), path
 * (cap) the path id.  Each path records at most one vertex per pass, at
 * most the first 2^20 / n_learned paths reaching a pass.  All buffers are
 * host memory owned by the caller.  MCRT_ERR_BOUNDS beyond 2^24 paths. */
MCRT_API int mcrt_debug_learned_records(mcrt_scene* scene, const mcrt_camera_desc* camera, uint64_t n, uint64_t seed,
                                        const mcrt_trace_opts* opts, int32_t cap, float* feat, float* dir,
                                        float* val, uint64_t* path, int32_t* count);

MCRT_API int mcrt_debug_pool_usage(mcrt_ctx* ctx, int32_t reset_high, uint64_t* used_current, uint64_t* used_high);

/* Philox4x32-10 evaluated on the device for n (counter[4], key[2]) pairs
 * (host arrays); out receives 4 words per pair. */
MCRT_API int mcrt_debug_philox(mcrt_ctx* ctx, const uint32_t* counters, const uint32_t* keys, uint32_t* out, size_t n);

#ifdef __cplusplus
}
#endif
#endif /* MCRT_H */
