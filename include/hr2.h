/*
 * hr2.h -- C ABI of the B300 (sm_103a) Helios-r2 emission forward model.
 *
 * The library evaluates, for a batch of parameter samples, the forward model
 * of Kitzmann et al. (2020), Sects. 2-3: finite-element temperature profile
 * (Sect. 2.5.1, Eqs. 12-16), opacity interpolation onto each level's (T, p)
 * and the abundance-weighted absorption coefficient (Sects. 2.3, 2.8), layer
 * optical depths, the scattering-free short-characteristic solve with a
 * linear Planck source over Gauss angle nodes (Sect. 2.1, Eqs. 1-8), the
 * radius-distance scaling (Sect. 2.2, Eq. 9), the Gaussian instrument
 * profile (Sect. 2.7, Eq. 17), binning to the observed bins (Sect. 2.8) and
 * the Gaussian log-likelihood with optional error inflation (Sect. 3.1
 * Eq. 19; Sect. 3.3 Eqs. 22-23).
 *
 * Conventions for every entry point
 *   - Return value: HR2_OK (0) or a negative hr2_status.  No C++ exception
 *     crosses the ABI.  hr2_last_error() gives a human-readable message for
 *     the calling thread's last failure on that context.
 *   - Device pointers are plain CUDA device addresses (e.g. a torch tensor's
 *     data_ptr()); host pointers are ordinary process memory.  Every argument
 *     says which it is.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Batch calls are asynchronous on that stream and do not
 *     synchronise the host, except where stated.
 *   - Ownership: the library owns contexts, tables and setups (create /
 *     destroy pairs); the caller owns every parameter and output buffer.
 *   - Units are cgs; wavenumbers in cm^-1; pressures in bar at the ABI.
 *   - Physically invalid samples (non-positive T on any level, f <= 0,
 *     d <= 0, absorber mixing ratios summing to >= 1, non-finite values)
 *     do not fail the call: their spectrum is NaN, their status word is
 *     non-zero and their log-likelihood is -inf.
 */
#ifndef HR2_H
#define HR2_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status */
typedef enum {
  HR2_OK = 0,
  HR2_EINVAL = -1,    /* invalid argument; nothing was launched           */
  HR2_ENOMEM = -2,    /* device allocation failed or memory budget hit    */
  HR2_ECUDA = -3,     /* a CUDA runtime call failed                       */
  HR2_ETIMEDOUT = -4, /* a bounded device-side wait gave up               */
  HR2_EBUSY = -5,     /* workspace cannot grow while the stream captures  */
  HR2_EBOUNDS = -6    /* a device-side index check failed (only in the
                         bounds-checked build, libhr2_bounds.so)          */
} hr2_status;

/* per-sample status bits written by forward_model_batch */
#define HR2_SAMPLE_BAD_T      1  /* a level temperature is <= 0 or not finite  */
#define HR2_SAMPLE_BAD_ABUND  2  /* mixing ratios sum to >= 1 or are not finite */
#define HR2_SAMPLE_BAD_SCALE  4  /* f, d or g not positive / finite            */
#define HR2_SAMPLE_BAD_SETUP  8  /* setup index outside [0, n_setups)          */
#define HR2_SAMPLE_BAD_CLOUD 16  /* cloud parameters not finite or f_c > 1     */

/* ---------------------------------------------------------------- limits */
#define HR2_MAX_TNODES   16   /* finite-element temperature nodes, K_e q + 1  */
#define HR2_MAX_SPECIES  16   /* absorbers per setup                          */
#define HR2_MAX_MU        8   /* Gauss angle nodes                            */
#define HR2_MAX_LEVELS  256   /* levels (layers + 1) per setup                */
#define HR2_MAX_SETUPS   32   /* distinct setups in one batch call            */
#define HR2_MAX_TGRID    64   /* points of a table's temperature grid         */
#define HR2_MAX_PGRID    64   /* points of a table's pressure grid            */

/* ------------------------------------------------ parameter vector layout
 * One row of HR2_NPARAM doubles per sample ("theta", Table 1 of the paper,
 * free-chemistry variant):
 *   [HR2_P_LOGG]      log10 g, g in cm s^-2
 *   [HR2_P_F]         calibration factor f of the radius-distance relation
 *   [HR2_P_DIST]      distance d in parsec; the FP16/FP32 path scales the
 *                     binned flux by f (R/d)^2 held as an FP32 head and tail,
 *                     so that factor must lie in FP32's normal range
 *                     (1.2e-38 .. 3.4e38; R < d gives at most f)
 *   [HR2_P_T0 + i]    finite-element nodal temperature i in K, i = 0 is the
 *                     bottom of the atmosphere (T_1 of Sect. 2.5.1); the setup
 *                     uses fe_elements*fe_order+1 of them
 *   [HR2_P_X0 + s]    log10 volume mixing ratio of the setup's absorber s
 *   [HR2_P_CLOUD]     gray cloud layer (setups with cloud != 0; Appendix,
 *                     "Impact of a gray cloud layer"): log10 of its optical
 *                     depth tau_c,
 *   [HR2_P_CLOUD + 1] log10 of its top pressure in bar,
 *   [HR2_P_CLOUD + 2] log10 f_c, 0 < f_c <= 1: the layer spans p_top to
 *                     p_top / f_c, tau_c spread evenly in pressure over it
 * With Milne's profile (HR2_PROFILE_MILNE) the temperature entries are
 *   [HR2_P_T0]        Tbar_eff in K (the gray-atmosphere parameter, Sect. 2.5)
 *   [HR2_P_T0 + 1]    log10 kappa_R, the Rosseland opacity in cm^2 g^-1
 * Unused entries are ignored.  hr2_nodes_from_b() converts (T_1, b_i) to
 * nodal temperatures. */
#define HR2_P_LOGG  0
#define HR2_P_F     1
#define HR2_P_DIST  2
#define HR2_P_T0    3
#define HR2_P_X0   19
#define HR2_P_CLOUD 35
#define HR2_NPARAM 38

/* ---------------------------------------------------------------- storage */
#define HR2_STORE_FP16_OFFSET 1  /* FP16 of (log10 sigma - off_s), off_s integer */
#define HR2_STORE_FP64        2  /* FP64 log10 sigma (the plain FP64 path)       */

/* hr2_setup_desc.level_cache: build the level-gridded operand where it fits */
#define HR2_LEVEL_CACHE_AUTO 2
/* hr2_setup_desc.level_cache: build the operand at every evaluation, one
 * group of tiles at a time, into a per-stream ring (see level_cache) */
#define HR2_LEVEL_CACHE_STREAM 3

/* Interpolation space of the opacity tables (Sect. 2.8 names the
 * interpolation of the tables but not the quantity interpolated). */
#define HR2_INTERP_LOG10  0  /* bilinear in log10 sigma, then 10^x (default)     */
#define HR2_INTERP_LINEAR 1  /* bilinear in sigma itself (CIA: linear in T)      */

/* Temperature profile (Sect. 2.5). */
#define HR2_PROFILE_FE    0  /* finite elements on Gauss-Lobatto nodes (Sect.
                                2.5.1; the default)                              */
#define HR2_PROFILE_MILNE 1  /* Milne's gray radiative-equilibrium profile
                                T^4 = 3/4 Tbar^4 [tau_R + q(tau_R)] with the
                                exact Hopf function q; tau_R = kappa_R p / g     */

/* Source-function interpolation of the short characteristics (Sect. 2.1). */
#define HR2_SC_LINEAR    0   /* linear between levels (Eqs. 4-7; the default)   */
#define HR2_SC_PARABOLIC 1   /* parabola through the level above, the level and
                                the level below (the top layer stays linear);
                                about twice the work per layer                  */

typedef struct hr2_ctx hr2_ctx;
typedef struct hr2_tables hr2_tables;
typedef struct hr2_setup hr2_setup;

/* Opacity table description (Sect. 2.3: per-species cross-sections tabulated
 * on a (T, p, nu) grid; CIA of H2-H2 and H2-He on (T, nu)).  All pointers
 * are HOST memory read during the call only. */
typedef struct {
  int n_species;              /* absorbers in the table, 1..HR2_MAX_SPECIES     */
  int n_T;                    /* 2..HR2_MAX_TGRID                               */
  const double* T_grid;       /* [n_T] K, strictly ascending, > 0               */
  int n_p;                    /* 2..HR2_MAX_PGRID                               */
  const double* log10p_grid;  /* [n_p] log10(p / bar), strictly ascending       */
  double nu0;                 /* wavenumber of column 0, cm^-1 (> 0)            */
  double dnu;                 /* uniform spacing, cm^-1 (> 0)                   */
  int n_nu;                   /* columns                                        */
  const double* species_mass; /* [n_species] molecular mass in u                */
  int has_cia_h2h2;           /* nonzero: an H2-H2 CIA table is supplied        */
  int has_cia_h2he;           /* nonzero: an H2-He CIA table is supplied        */
} hr2_table_desc;

/* Spectral / atmospheric setup (Sects. 2, 2.1, 2.5.1, 2.7).  Pointers are
 * HOST memory read during the call only. */
typedef struct {
  int nu_first;               /* first table column used                        */
  int n_nu;                   /* columns used (>= 1)                            */
  int n_layers;               /* L layers; L+1 levels equidistant in log p      */
  double p_top, p_bot;        /* bar, 0 < p_top < p_bot                         */
  int n_species;              /* absorbers used, 0..HR2_MAX_SPECIES             */
  const int* species;         /* [n_species] table indices                      */
  int n_mu;                   /* Gauss-Legendre angle nodes, 1..HR2_MAX_MU      */
  int fe_elements;            /* K_e >= 1                                       */
  int fe_order;               /* q >= 1, K_e q + 1 <= HR2_MAX_TNODES            */
  double resolving_power;     /* R = nu / FWHM of the instrument; <= 0: none    */
  int n_bins;                 /* >= 1; every bin must contain a grid point     */
  const double* bin_edges;    /* [n_bins+1] cm^-1 ascending; a point nu belongs
                                 to bin b if edge_b <= nu < edge_{b+1} (last bin
                                 closed)                                         */
  const double* obs_flux;     /* [n_bins] observed D_j, or NULL                 */
  const double* obs_sigma;    /* [n_bins] observational errors sigma_j, or NULL */
  double r_he;                /* n_He / n_H2 of the H2/He filling gas (> 0)     */
  double radius_cm;           /* R_* of the radius-distance relation, cm        */
  int level_cache;            /* FP16 tables only.  Nonzero: interpolate the
                                 tables in p onto this setup's levels once, at
                                 creation (FP64 arithmetic, stored as FP32
                                 times log2 10: per T cell the row and its
                                 difference to the next T row, n_species x
                                 levels x (n_T - 1) x columns x 8 bytes of
                                 device memory), so that each sample
                                 interpolates in T only.  Zero:
                                 every evaluation interpolates the FP16 tables
                                 bilinearly.  HR2_LEVEL_CACHE_AUTO: the
                                 operand if it fits both the context's budget
                                 (when one is set) and half the device's free
                                 memory at creation, else the streamed operand
                                 below (the linear option, which needs the
                                 operand, then fails with HR2_ENOMEM).  hr2_setup_memory
                                 tells which was built.  One batch call takes
                                 setups of a single kind.
                                 HR2_LEVEL_CACHE_STREAM (log10 option only):
                                 no operand is kept; a call of at least 32
                                 samples whose setups are all streamed builds
                                 their operands per group of consecutive
                                 128-point tiles (only the level and T cell
                                 blocks its samples use) into a ring in the
                                 stream's workspace
                                 (FP32 arithmetic; at most 4 GiB unless
                                 hr2_set_stream_group says otherwise) and
                                 sweeps each group before the next is built,
                                 which costs one operand build per call but
                                 holds only the ring on the device; smaller
                                 calls and calls that mix it with setups of
                                 another kind read the tables directly, and
                                 so does a call
                                 whose ring fits neither the context's budget
                                 nor the device's memory.  The ring and the
                                 group descriptors are allocated by a call on
                                 the stream that needs more than it holds,
                                 never during stream capture: capture a
                                 streamed batch only after one eager call of
                                 the same size on that stream (HR2_EBUSY
                                 otherwise).  hr2_setup_memory
                                 reports HR2_LEVEL_CACHE_STREAM for it.          */
  int interp;                 /* HR2_INTERP_LOG10 or HR2_INTERP_LINEAR.  With
                                 FP16 tables the linear option needs
                                 level_cache (the operand then holds the
                                 p-interpolated cross-sections, so each sample
                                 interpolates in T with FMAs only); FP64
                                 tables take either.  One batch call takes
                                 setups of a single option.                      */
  int profile;                /* HR2_PROFILE_FE or HR2_PROFILE_MILNE.  Milne's
                                 profile tabulates q(tau) once at creation
                                 (Chandrasekhar's H-function representation,
                                 FP64; 32 KB of device memory); a batch may mix
                                 profiles.                                       */
  int cloud;                  /* nonzero: add the gray cloud layer of
                                 parameters HR2_P_CLOUD.. (its optical depth is
                                 the same at every wavenumber and adds to the
                                 layers' absorption optical depths)              */
  int sc;                     /* HR2_SC_LINEAR or HR2_SC_PARABOLIC.  One batch
                                 call takes setups of a single kind.             */
} hr2_setup_desc;

/* Launch shape of the persistent forward kernel: the work item's tile
 * (samples x wavenumbers), the persistent grid and the copy-pipeline depth
 * (chosen by the autotuner; a new context starts with {2, 8, 1, 0, 2}).  Every
 * shape computes each (sample, wavenumber) the same way: results do not
 * depend on it. */
typedef struct {
  int warps_per_cta;          /* samples processed together per work item: 1..16;
                                 a batch with fewer samples uses fewer, with
                                 proportionally more CTAs per SM               */
  int ctas_per_sm;            /* persistent CTAs per SM: 1..32                    */
  int tiles_per_item;         /* consecutive 128-point wavenumber tiles per work
                                 item, 1..16 (the item's wavenumber extent)     */
  int stages;                 /* shared-memory stages per warp of the level-
                                 gridded kernel: 0 = by batch shape; 1 or 2
                                 where the kernel exists in both depths (more
                                 than 4 angle nodes, 8 or more absorbers, linear
                                 source), else the batch-shape choice stands    */
  int split_max_batch;        /* setups read from the FP16 tables in place
                                 (no level-gridded operand), linear source:
                                 batches of at most this many samples run in
                                 two passes -- every level's absorption
                                 coefficient first, one warp per (sample, level,
                                 tile), then the level sweep -- which keeps many
                                 more table reads in flight; same results bit
                                 for bit, n x levels x columns x 4 bytes of
                                 workspace; 0 = never, at most 65535            */
} hr2_launch_cfg;

/* ------------------------------------------------------------- contexts */

/* Create a context on CUDA device `device`.  mem_budget_bytes caps the
 * device memory the context may hold for tables, setups and workspace
 * (0 = no cap beyond the device).  *out receives the handle. */
int hr2_ctx_create(int device, size_t mem_budget_bytes, hr2_ctx** out);

/* Destroy a context and every table, setup and workspace it still owns.
 * The caller must have finished all work it launched with it. */
int hr2_ctx_destroy(hr2_ctx* ctx);

/* Message of the calling thread's last failure on ctx ("" if none).  The
 * string is owned by the library and valid until the next call on ctx. */
const char* hr2_last_error(const hr2_ctx* ctx);

/* Device bytes currently held by ctx and its budget (0 = uncapped). */
int hr2_ctx_memory(const hr2_ctx* ctx, size_t* used_bytes, size_t* budget_bytes);

/* Set / read the persistent kernel's launch shape used by later calls. */
int hr2_set_launch_config(hr2_ctx* ctx, const hr2_launch_cfg* cfg);
int hr2_get_launch_config(const hr2_ctx* ctx, hr2_launch_cfg* cfg);

/* Make sure the workspace of `stream` holds a batch of n samples whose
 * setups span at most n_nu_max wavenumbers, so that a later batch call of
 * that size allocates nothing (required before CUDA-graph capture). */
int hr2_reserve(hr2_ctx* ctx, void* stream, int n, int n_nu_max);

/* -------------------------------------------------------------- tables */

/* create_opacity_tables: copy the cross-section tables to the device and
 * keep them resident (Sects. 2.3, 2.8).
 *   log10_sigma     HOST [n_species][n_T][n_p][n_nu] log10 sigma in cm^2, or
 *                   NULL to upload each species later with
 *                   hr2_tables_upload_species();
 *   log10_cia_h2h2  HOST [n_T][n_nu] log10 k in cm^5, or NULL (required iff
 *                   desc->has_cia_h2h2); log10_cia_h2he likewise;
 *   storage         HR2_STORE_FP16_OFFSET: each species s (and each CIA
 *                   table) is stored as IEEE binary16 of (value - off_s),
 *                   rounded to nearest even, with off_s = rint((min+max)/2)
 *                   over that species' values; HR2_STORE_FP64: stored as is.
 * All values must be finite.  The wavenumber axis is padded on the device to
 * a multiple of 64 columns.  *out receives the handle. */
int create_opacity_tables(hr2_ctx* ctx, const hr2_table_desc* desc, const double* log10_sigma,
                          const double* log10_cia_h2h2, const double* log10_cia_h2he, int storage,
                          hr2_tables** out);

/* Upload (or replace) species s: HOST [n_T][n_p][n_nu] log10 sigma.  Lets
 * large tables be filled one species at a time.  Synchronous. */
int hr2_tables_upload_species(hr2_ctx* ctx, hr2_tables* tables, int s, const double* log10_sigma_s);

/* Offsets off_s (HOST [n_species + 2] out: species, then H2-H2, H2-He CIA)
 * and device bytes of the stored table. */
int hr2_tables_info(const hr2_tables* tables, double* offsets_out, size_t* device_bytes);

int hr2_tables_destroy(hr2_ctx* ctx, hr2_tables* tables);

/* --------------------------------------------------------------- setups */

/* Build a setup on the device: level grid, Gauss-Legendre angle nodes,
 * Gauss-Lobatto element nodes, per-level pressure interpolation weights and
 * the combined instrument-profile + binning operator W (a banded sparse
 * matrix, FP32 and FP64, Sects. 2.7-2.8), plus the observation if given.
 * Synchronous.  The tables must outlive the setup. */
int hr2_setup_create(hr2_ctx* ctx, const hr2_tables* tables, const hr2_setup_desc* desc, hr2_setup** out);

/* Replace the observation (HOST [n_bins] each; D finite, sigma > 0, else
 * HR2_EINVAL).  Also precomputes on the device the likelihood's terms that do
 * not depend on the model (1 / (2 sigma^2) per bin and the normalisation
 * sum_b -ln(2 pi sigma_b^2) / 2 of Eq. 19), used when a sample has no error
 * inflation.  Device memory: (3 n_bins + 1) doubles.  Synchronous. */
int hr2_setup_set_observation(hr2_ctx* ctx, hr2_setup* setup, const double* obs_flux, const double* obs_sigma);

/* Number of bins / wavenumbers / nonzeros of W of a setup. */
int hr2_setup_info(const hr2_setup* setup, int* n_bins, int* n_nu, long long* w_nnz);

/* Device bytes a setup holds (levels, quadratures, W, observation, Hopf table,
 * wavenumber constants and, if built, the level-gridded operand), the
 * operand's share of them, and whether the operand was built (1) or the
 * setup evaluates the FP16 tables directly (0).  No counterpart in the
 * paper.  NULL outputs are skipped. */
int hr2_setup_memory(const hr2_setup* setup, size_t* bytes, size_t* operand_bytes, int* level_gridded);

int hr2_setup_destroy(hr2_ctx* ctx, hr2_setup* setup);

/* ----------------------------------------------------------- batch calls */

/* forward_model_batch: model spectra of n samples (Sects. 2.1-2.8).
 *   setups           HOST [n_setups] handles, 1 <= n_setups <= HR2_MAX_SETUPS;
 *                    all must share one table set and one storage type
 *   setup_of_sample  DEVICE int [n]: index into `setups` per sample
 *   params           DEVICE double [n][HR2_NPARAM] (layout above)
 *   out_bins         DEVICE float [n][bins_ld]: D_m of sample i in its first
 *                    n_bins entries (FP32), scaled by f (R_star/d)^2
 *   out_highres      DEVICE float [n][highres_ld] or NULL: unscaled top-of-
 *                    atmosphere flux F+ (Eq. 8) on the setup's n_nu points
 *   out_status       DEVICE int [n] or NULL: HR2_SAMPLE_* bits per sample
 * FP16-offset tables run the FP32 persistent kernel; FP64 tables run the
 * plain FP64 kernel.  Results for a sample do not depend on the rest of the
 * batch.  Asynchronous on `stream`; uses the stream's workspace. */
int forward_model_batch(hr2_ctx* ctx, int n_setups, const hr2_setup* const* setups,
                        const int* setup_of_sample, const double* params, int n, float* out_bins,
                        int bins_ld, float* out_highres, int highres_ld, int* out_status, void* stream);

/* log_likelihood_batch: Gaussian log-likelihood (Eq. 19), with error
 * inflation s_j^2 = sigma_j^2 + 10^eps (Eqs. 22-23) where log_eps[i] is
 * finite.  FP64 accumulation in a fixed order (deterministic).
 *   model_bins   DEVICE float [n][bins_ld] (as written by forward_model_batch)
 *   log_eps      DEVICE double [n] or NULL (NULL or NaN: no inflation)
 *   out_lnL      DEVICE double [n]; -inf where any model bin is not finite
 * Every setup used must have an observation.  Asynchronous on `stream`. */
int log_likelihood_batch(hr2_ctx* ctx, int n_setups, const hr2_setup* const* setups,
                         const int* setup_of_sample, const float* model_bins, int bins_ld,
                         const double* log_eps, int n, double* out_lnL, void* stream);

/* hr2_evaluate_host: the call a sampler makes per batch of live points, with
 * HOST buffers: copies setup_of_sample (int [n]), params (double
 * [n][HR2_NPARAM]) and log_eps (double [n] or NULL) to the stream's
 * workspace, runs forward_model_batch and log_likelihood_batch, and copies
 * lnL (double [n]) and, if out_bins is not NULL, the model bins (float
 * [n][bins_ld]) back.  Synchronises `stream` before returning.  Pinned host
 * buffers make the copies asynchronous with respect to other streams. */
int hr2_evaluate_host(hr2_ctx* ctx, int n_setups, const hr2_setup* const* setups,
                      const int* setup_of_sample, const double* params, const double* log_eps, int n,
                      double* out_lnL, float* out_bins, int bins_ld, void* stream);

/* ------------------------------------------------- allocation-free variant
 * (No counterpart in the paper.)  forward_model_batch_noalloc computes
 * exactly what forward_model_batch computes, for FP16-offset tables, but
 * allocates no device memory at all.  It is for callers that may not let a
 * library allocate: a host application whose device memory belongs to
 * another allocator (a framework's caching pool that must account for every
 * byte), or a latency-critical evaluation loop that cannot accept the
 * device-wide synchronisation cudaMalloc may imply.  A setup created with
 * HR2_LEVEL_CACHE_STREAM (or streamed by HR2_LEVEL_CACHE_AUTO) is read
 * directly here at every batch size, since its ring would need an
 * allocation: from 32 samples up forward_model_batch streams it instead, and
 * the two agree to the FP32 rounding of the streamed operand.
 *
 * Its scratch (per-sample and per-level records, the work plan and the work
 * counter) lives in one statically sized device array of
 * HR2_NOALLOC_SCRATCH_BYTES, which every GPU that loads the library holds
 * until the process exits.  The caller passes all inputs and outputs as for
 * forward_model_batch, except that out_highres is REQUIRED: the F+ buffer is
 * an output here, not scratch.
 *   - Limit: the batch must fit the array, roughly n * (L+1) * 64 bytes plus
 *     n * 220 bytes plus 1 KB (about 1024 samples of 121 levels); larger
 *     batches, FP64 tables or a NULL out_highres return HR2_EINVAL with a
 *     message giving the bytes needed.
 *   - The first call on a device looks up the array's device address (once
 *     per device, with that device current); make that first call before any
 *     stream capture.
 *   - All calls share the one array and it keeps the last call's contents;
 *     the work counter that must start at zero is cleared on the device by
 *     each call itself.  Calls whose work overlaps on the GPU (different
 *     streams, or different host threads) race on the array: serialise them. */
#define HR2_NOALLOC_SCRATCH_BYTES (8u << 20)
int forward_model_batch_noalloc(hr2_ctx* ctx, int n_setups, const hr2_setup* const* setups,
                                const int* setup_of_sample, const double* params, int n, float* out_bins,
                                int bins_ld, float* out_highres, int highres_ld, int* out_status, void* stream);

/* -------------------------------------------------------- instrumentation
 * (No counterpart in the paper.)  While enabled, every forward_model_batch
 * records a pair of CUDA events on its stream around the launch of the main
 * forward kernel (k_forward32 / k_forward64; with the two-pass direct path,
 * around both passes; with the streamed operand, around every group's
 * build, plan and sweep), so a caller can time that
 * kernel alone inside a longer step.  hr2_profile_read waits for the
 * recorded events, returns the summed kernel time in ms and the number of
 * launches, and with reset != 0 forgets them. */
int hr2_profile_enable(hr2_ctx* ctx, int on);
int hr2_profile_read(hr2_ctx* ctx, int reset, double* kernel_ms, int* launches);

/* hr2_measure_unit_rate: (No counterpart in the paper.)  Throughput of one
 * arithmetic unit of `device`, measured by a microbenchmark kernel at full
 * occupancy (8 CTAs of 256 threads per SM, 16 independent dependency chains
 * per thread, `iters` steps per chain, one warm-up launch of iters/16 steps
 * first).  These are the denominators of the forward kernel's roofline:
 *   HR2_UNIT_EX2_RCP  half the chains y <- 2^(-y), half y <- 1/y + 1: the
 *                     two special functions interleaved (ops counts both)
 *   HR2_UNIT_RCP      y <- 1/y + 1, rcp.approx.ftz and an FP32 addition
 *   HR2_UNIT_EX2      y <- 2^(-y), ex2.approx.ftz after an FP32 negation
 *   HR2_UNIT_FFMA     scalar FP32 fused multiply-add
 *   HR2_UNIT_FFMA2    packed f32x2 fused multiply-add (ops counts
 *                     instructions, each two FMAs)
 * `out` (HOST) receives the CUDA-event time, the operations, operations per
 * second, operations per SM cycle (the cycles being the median over SMs of the
 * span from an SM's first CTA start to its last CTA end, in that SM's
 * clock64) and the SM clock those cycles imply over the event time.  Synchronous;
 * allocates and frees its own small buffers.  Returns HR2_EINVAL for an
 * unknown kind or iters < 1, HR2_ECUDA on a CUDA error. */
#define HR2_UNIT_EX2_RCP 0
#define HR2_UNIT_RCP 1
#define HR2_UNIT_EX2 2
#define HR2_UNIT_FFMA 3
#define HR2_UNIT_FFMA2 4
#define HR2_UNIT_KINDS 5
typedef struct {
  double ms;              /* kernel time (CUDA events)                     */
  double ops;             /* operations executed                           */
  double ops_per_s;
  double sm_ghz;          /* SM cycles of the run / event time             */
  double ops_per_clk_sm;  /* ops / n_sm / SM cycles of the run (median SM) */
  int n_sm;
} hr2_unit_rate;
int hr2_measure_unit_rate(int device, int kind, long long iters, hr2_unit_rate* out);

/* Wait for `stream` and report whether a bounded device-side wait of the
 * last batch on that stream gave up (HR2_ETIMEDOUT; its outputs are then not
 * valid).  No counterpart in the paper.  hr2_evaluate_host checks the same
 * word itself. */
int hr2_stream_check(hr2_ctx* ctx, void* stream);

/* hr2_noalloc_check: the same report for forward_model_batch_noalloc, whose
 * error word lives in the shared static array: waits for `stream`, then
 * reads the word the last allocation-free call (on any stream of this
 * device) left.  A 4-byte device-to-host copy; allocates nothing.  No
 * counterpart in the paper. */
int hr2_noalloc_check(hr2_ctx* ctx, void* stream);

/* Tiles per group of the streamed operand (HR2_LEVEL_CACHE_STREAM) for
 * later calls: 0 (the default) sizes each group so that it holds about eight
 * work items per persistent CTA, with the ring at most 4 GiB; a positive
 * count fixes it (the ring then holds that many tiles' operand, which the
 * context's budget must allow).  No counterpart in the paper: it trades the
 * ring's memory against the number of groups.  HR2_EINVAL for tiles < 0. */
int hr2_set_stream_group(hr2_ctx* ctx, int tiles);

/* hr2_set_wait_limit / hr2_get_wait_limit: SM clock cycles (>= 0) that a
 * device-side pipeline wait of the forward kernel may take before it gives
 * up; default 2e9 (about 1 s).  A wait that gives up sets the batch's error
 * word (HR2_ETIMEDOUT from hr2_stream_check, hr2_evaluate_host or
 * hr2_noalloc_check), waits again for its own copies to land (as long as the
 * limit, and at least 1e7 cycles) and stops its warp; the batch's outputs
 * are then not valid, and the next batch starts from a clean state.  The
 * limit applies to batches launched after the call.  No counterpart in the
 * paper.  HR2_EINVAL for cycles < 0. */
int hr2_set_wait_limit(hr2_ctx* ctx, long long cycles);
int hr2_get_wait_limit(const hr2_ctx* ctx, long long* cycles);

/* hr2_set_wait_fault: test hook for the path above (no counterpart in the
 * paper).  While on, the level-gridded forward kernel arms the barrier of each
 * work item's first pipeline stage for 16 bytes more than its copies deliver:
 * a flag that nothing sets, so that the stage's wait runs out after the wait
 * limit every time (its copies still land; the drain then waits at least
 * ~1e7 cycles for them).  Nothing faults, traps or hangs; the batch reports
 * HR2_ETIMEDOUT.  Off by default; a context's later batches are unaffected
 * once it is off again. */
int hr2_set_wait_fault(hr2_ctx* ctx, int on);

/* hr2_effective_temperature: T_eff of each sample (Sect. 2.6): its F+ (the
 * high-resolution output of forward_model_batch, before the distance
 * dilution of Eq. 9) integrated over its setup's wavenumber grid by the
 * trapezoid rule in FP64, converted by the Stefan-Boltzmann law F = sigma
 * T_eff^4.  Meaningful for a setup spanning the emitted spectrum (the paper
 * integrates 1-20 micron).  DEVICE pointers: setup_of_sample int [n],
 * highres float [n][highres_ld] (as forward_model_batch wrote it), out_teff
 * double [n] (NaN for a sample with an invalid setup index or NaN flux).
 * Asynchronous on `stream`. */
int hr2_effective_temperature(hr2_ctx* ctx, int n_setups, const hr2_setup* const* setups, const int* setup_of_sample,
                              const float* highres, int highres_ld, int n, double* out_teff, void* stream);

/* ------------------------------------------------------ nested sampling
 * Evidence bookkeeping of nested sampling (Sect. 3.2, after Skilling 2004),
 * kept on the device so that a sampler can run propose -> forward_model_batch
 * -> log_likelihood_batch -> hr2_ns_absorb on one stream without a host
 * round trip per replacement.  With N live points the i-th point to leave
 * the live set (the lowest likelihood, L*_i) has prior mass X_i = exp(-i/N)
 * inside its contour and shell weight w_i = X_{i-1} - X_i (X_0 = 1);
 * ln Z = ln sum_i L*_i w_i and the information H = sum_i p_i ln(L*_i / Z),
 * p_i = L*_i w_i / Z, accumulate in FP64 log-sum-exp: each absorb call
 * folds its dead points into the running (ln Z, H) with a fixed-order warp
 * reduction (the closed form of adding them one at a time; equal to
 * rounding, deterministic).  The sampler itself (MultiNest in the paper) is the
 * caller's; this is the part that runs per likelihood batch. */
typedef struct {
  long long n_dead;   /* dead points so far (i of the last one)              */
  long long n_seen;   /* candidates examined so far                          */
  double log_z;       /* ln Z over the dead points; -inf before the first    */
  double info;        /* H over the dead points, nats                        */
  double log_x;       /* ln X of the last dead point, -n_dead / N            */
  double lnl_min;     /* smallest live lnL after the call                    */
  double lnl_max;     /* largest live lnL after the call                     */
  double reserved;
} hr2_ns_state;

/* hr2_ns_state_init: a fresh state (n_dead 0, log_z -inf, H 0) in the DEVICE
 * struct `state`, asynchronously on `stream`. */
int hr2_ns_state_init(hr2_ctx* ctx, hr2_ns_state* state, void* stream);

/* hr2_ns_absorb: use n_cand scored candidates in order (Sect. 3.2): a
 * candidate with lnL strictly above the live minimum (ties: lowest index; a
 * NaN counts as +inf) replaces that live point, which becomes dead point i =
 * n_dead + 1 with ln w_i = -(i-1)/N + ln(1 - e^(-1/N)); other candidates are
 * skipped.  Stops when dead_cap dead points exist (the rest are not
 * examined; state->n_seen tells how far it got).  All pointers are DEVICE:
 *   live_lnl     double [n_live], live_theta double [n_live][HR2_NPARAM]
 *                (updated in place)
 *   cand_lnl     double [n_cand], cand_theta double [n_cand][HR2_NPARAM]
 *   state        hr2_ns_state (updated; lnl_min / lnl_max refreshed)
 *   dead_lnl, dead_logw  double [dead_cap], dead_theta double
 *                [dead_cap][HR2_NPARAM]: dead point k at index k (absolute)
 * Asynchronous on `stream`; one warp (the candidates are consumed in
 * order).  Returns HR2_EINVAL for n_live < 1, n_cand < 0 or NULL pointers. */
int hr2_ns_absorb(hr2_ctx* ctx, int n_live, double* live_lnl, double* live_theta, int n_cand, const double* cand_lnl,
                  const double* cand_theta, hr2_ns_state* state, double* dead_lnl, double* dead_logw,
                  double* dead_theta, long long dead_cap, void* stream);

/* hr2_ns_propose: candidates for the next round of a minimal nested sampler
 * (a stand-in for MultiNest's ellipsoidal proposals, Sect. 3.2), drawn on the
 * device: uniform in the bounding box of the live points, widened by
 * `enlarge` x its span on each side and clipped to the prior box [prior_lo,
 * prior_hi]; a parameter with prior_lo == prior_hi stays at prior_lo.  Uniform
 * deviates: SplitMix64 (Steele, Lea & Flood 2014) of (seed, counter + i *
 * HR2_NPARAM + p), so a call consumes n * HR2_NPARAM counter values and equal
 * arguments give equal draws.  All pointers are DEVICE:
 *   live_theta          double [n_live][HR2_NPARAM]
 *   prior_lo, prior_hi  double [HR2_NPARAM]
 *   box                 double [HR2_NPARAM][2] (written: the proposal box)
 *   out_theta           double [n][HR2_NPARAM] (written)
 * Asynchronous on `stream`.  Returns HR2_EINVAL for n_live < 1, n < 0,
 * enlarge < 0 (or NaN) or NULL pointers. */
int hr2_ns_propose(hr2_ctx* ctx, int n_live, const double* live_theta, const double* prior_lo,
                   const double* prior_hi, double enlarge, int n, double* box, double* out_theta,
                   unsigned long long seed, unsigned long long counter, void* stream);

/* hr2_ns_finalize: ln Z and H with the live points added, each with weight
 * X_n / N (fixed-order reduction): out (DEVICE double [2]) = {ln Z, H}.  The state
 * is not modified.  Asynchronous on `stream`. */
int hr2_ns_finalize(hr2_ctx* ctx, int n_live, const double* live_lnl, const hr2_ns_state* state, double* out,
                    void* stream);

/* ------------------------------------------------------------- helpers */

/* Nodal temperatures from the retrieved bottom temperature T_1 and the
 * ratios b_i (Sect. 2.5.1): node i+1 = b_i * node i.  HOST arrays:
 * b [n_nodes-1], nodes_out [n_nodes]. */
int hr2_nodes_from_b(int n_nodes, double T1, const double* b, double* nodes_out);

/* Library version string. */
const char* hr2_version(void);

#ifdef __cplusplus
}
#endif
#endif /* HR2_H */
