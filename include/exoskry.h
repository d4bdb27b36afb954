/*
 * exoskry.h - C ABI of the GB300-native batched forward model, Gaussian
 * log-likelihood and adjoint for sub-stellar atmospheric retrieval
 * (Exo Skryer, arXiv 2602.19687).
 *
 * The problem statement the calls follow (Sect. 2, 2.3): a sampler proposes
 * parameter vectors theta; the library evaluates the forward model spectrum
 * for each vector and its Gaussian log-likelihood against binned data
 * (Eq. lnL with residuals r_i and the error inflation of Eq. c_error);
 * invalid forward-model output is assigned ln L = -1e300.
 *
 * Conventions shared by every entry point:
 *  - Units are cgs; pressures in the API are in bar, wavelengths in micron,
 *    wavenumbers in cm^-1.
 *  - A context owns every device copy it makes (tables, grids, data, batch,
 *    workspace). Host inputs are copied during the call; the caller keeps
 *    ownership of its memory.
 *  - `mem` arguments say where a caller buffer lives: ES_MEM_HOST (pageable
 *    or pinned host memory; the call copies through the device and
 *    synchronises `stream` before returning) or ES_MEM_DEVICE (device memory
 *    of the context's GPU; the call is asynchronous on `stream`).
 *  - `stream` is a cudaStream_t passed as void*; NULL is the legacy default
 *    stream.
 *  - Errors are returned as es_status; es_last_error() gives a message.
 *    An invalid sample is not an error (it gets ln L = -1e300, zero
 *    gradient and flag bit ES_FLAG_INVALID).
 *  - One context must not be used from two host threads at once.
 */
#ifndef EXOSKRY_H
#define EXOSKRY_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct es_ctx es_ctx;
typedef void *es_stream_t;

typedef enum {
    ES_OK = 0,
    ES_EINVAL = 1,    /* bad argument, size or inconsistent description  */
    ES_ENOMEM = 2,    /* device or host allocation failed                */
    ES_ECUDA = 3,     /* a CUDA runtime call or kernel launch failed     */
    ES_ESTATE = 4,    /* call out of order (e.g. forward before tables)  */
    ES_ETIMEOUT = 5   /* a bounded device-side wait gave up              */
} es_status;

enum { ES_TP_ISOTHERMAL = 0, ES_TP_GUILLOT = 1, ES_TP_GUILLOT_MOD = 2, ES_TP_MILNE = 3 };
/* Emission output: planet-to-star flux ratio (Sect. 5, Fp/F*) or the
 * absolute flux of an isolated brown dwarf at distance D (Sect. 5, F_bd). */
enum { ES_FLUX_PLANET_STAR = 0, ES_FLUX_BROWN_DWARF = 1 };
enum { ES_CLOUD_NONE = 0, ES_CLOUD_DECK = 1, ES_CLOUD_KH18 = 2 };
/* Vertical profile of the non-grey cloud's mass mixing ratio (Sect. 2.5.1),
 * evaluated at each layer's pressure p:
 *   ES_QC_POWER_LAW  q_base (p / p_base)^alpha_c for p <= p_base, 0 below
 *   ES_QC_SLAB       q_slab at every pressure
 *   ES_QC_SLAB_BAND  q_slab for p_top <= p <= p_top + dp, 0 elsewhere */
enum { ES_QC_POWER_LAW = 0, ES_QC_SLAB = 1, ES_QC_SLAB_BAND = 2 };
/* Angles of the emergent-flux integral F = 2 pi int_0^1 I(mu) mu dmu (Sect. 5):
 *   ES_QUAD_GAUSS_LEGENDRE  4-point Gauss-Legendre on [0, 1], F = 2 pi sum w_j mu_j I_j
 *   ES_QUAD_GAUSS_JACOBI    4-point Gauss-Jacobi rule of the weight mu on [0, 1]
 *                           ("8-stream": 4 angles per hemisphere), F = 2 pi sum W_j I_j */
enum { ES_QUAD_GAUSS_LEGENDRE = 0, ES_QUAD_GAUSS_JACOBI = 1 };
/* Emission solver (Sect. 5):
 *   ES_RT_ABSORPTION  linear-in-tau Schwarzschild integration without
 *                     scattering (Rayleigh extinction counted as absorption)
 *   ES_RT_DELTA_EAA   the paper's delta-M scaled extended absorption
 *                     approximation, linear in tau. The paper cites the scheme
 *                     without its formulas; this library's reading: H2/He
 *                     Rayleigh scatters (albedo 1, asymmetry 0) and the
 *                     non-grey cloud scatters with the model constants
 *                     cloud_ssa and cloud_g; delta-M scaling with the forward
 *                     fraction f = g^2 of the layer's scattering-weighted
 *                     asymmetry g; zeroth order: absorption-only RT in both
 *                     directions on the scaled absorption depth; then one
 *                     upward pass on the full scaled depth with the source
 *                     (1 - w') B + w' (J + 3 g' mu H) of that field's mean
 *                     intensity J and flux moment H. Cloud kinds NONE or KH18. */
enum { ES_RT_ABSORPTION = 0, ES_RT_DELTA_EAA = 1 };
enum { ES_KIND_TRANSMISSION = 0, ES_KIND_EMISSION = 1 };
enum { ES_TABLE_F32 = 0, ES_TABLE_BF16 = 1 };
enum { ES_MEM_HOST = 0, ES_MEM_DEVICE = 1 };
/* Per-sample flags (es_get_flags): ES_FLAG_INVALID the sample's ln L is
 * -1e300 (invalid forward-model output, Sect. 2.3); ES_FLAG_TIMEOUT a kernel
 * of the call gave up on a bounded device-side wait, so every sample of that
 * call is invalid (set together with ES_FLAG_INVALID). */
enum { ES_FLAG_INVALID = 1, ES_FLAG_TIMEOUT = 2 };

/*
 * Canonical parameter vector. Slots 0..S-1 hold log10 of the S absorber
 * volume mixing ratios (Sect. 3.1); the slots below follow at S + ES_P_*.
 *   T_ISO        isothermal temperature [K]                  (Sect. 2.4.1)
 *   T_INT, T_EQ  internal / equilibrium temperature [K]     (Sect. 2.4.4)
 *   LOG_KAPPA_IR log10 infrared opacity [cm^2 g^-1]          (Sect. 2.4.3)
 *   LOG_GAMMA_V  log10 visible-to-infrared opacity ratio     (Sect. 2.4.4)
 *   Q_IRR0, LOG_P_T, BETA  stretched-exponential Hopf function
 *                of the irradiation term, Eq. (q); p_t in bar (GUILLOT_MOD);
 *                LOG_P_T and BETA also parameterise the MILNE Hopf function
 *   LOG_G        log10 reference gravity [cm s^-2]
 *   R_P          planet radius at p_ref [Jupiter radii, 7.1492e9 cm]
 *                (unused with ES_FLUX_BROWN_DWARF: the radius is derived)
 *   LOG_P_CLOUD  log10 grey cloud-deck pressure [bar]        (ES_CLOUD_DECK)
 *   C_INFL       error inflation c of Eq. c_error (-99: none)
 *   DILUTION     dilution factor s of Sect. 5 (emission)
 *   T_RATIO      skin-to-internal temperature ratio T_skin/T_int of the
 *                modified Milne profile, q0 = 4/3 T_RATIO^4 (Sect. 2.4.3)
 *   M_BD         brown-dwarf mass [Jupiter masses, 1.89813e30 g]; the radius
 *                is R_bd = sqrt(G M_bd / g) (Sect. 5, ES_FLUX_BROWN_DWARF)
 * Non-grey cloud (ES_CLOUD_KH18, Sect. 2.5): extinction rho_a kappa_ext with
 * kappa_ext = 3 q_c^eff Q_ext(x) / (4 r_eff), Q_ext = 1/(Q0 x^-a + x^0.2),
 * x = 2 pi r_eff nu, q_c^eff(p) = q_base (p/p_base)^alpha_c above the base
 * (0 below; or one of the slab profiles of cloud_profile), and the cloud
 * fraction f_cld mixing cloudy and clear spectra:
 *   LOG_QC       log10 q_base (effective mass mixing ratio at the base), or
 *                log10 q_slab of the slab profiles
 *   LOG_PC_BASE  log10 cloud-base pressure [bar]
 *   ALPHA_C      power-law index alpha_c of q_c^eff above the base
 *   LOG_R_EFF    log10 effective particle radius [micron]
 *   A_KH         spectral slope index a of Q_ext
 *   LOG_Q0       log10 Q0 of Q_ext
 *   F_CLD        cloud fraction f_cld in [0, 1]
 *   LOG_PC_TOP   log10 p_top of the slab band [bar]            (ES_QC_SLAB_BAND)
 *   LOG_DPC      log10 of the band's pressure extent dp [bar]  (ES_QC_SLAB_BAND)
 * The band's edges decide which layers hold cloud, so lnL is piecewise
 * constant in LOG_PC_TOP and LOG_DPC: their gradient is zero.
 * Mid-infrared feature (cloud_feature = 1, Sect. 2.5.3): Q_ext = min(Q_cont +
 * W(x) Q_feat, 2) with W = exp(-x / 0.5), Q_feat = 2 A exp(-z^2/2) Phi(xi z),
 * z = (lambda - lambda_0) / omega, Phi the standard normal CDF, lambda in
 * micron, the cap applied to Q_ext / Q_1 (Q_1 folded into q_c^eff):
 *   FEAT_A       peak amplitude A
 *   FEAT_LAM0    central wavelength lambda_0 [micron]
 *   FEAT_W       width omega [micron]
 *   FEAT_XI      skewness xi
 */
enum {
    ES_P_T_ISO = 0, ES_P_T_INT, ES_P_T_EQ, ES_P_LOG_KAPPA_IR, ES_P_LOG_GAMMA_V,
    ES_P_Q_IRR0, ES_P_LOG_P_T, ES_P_BETA, ES_P_LOG_G, ES_P_R_P, ES_P_LOG_P_CLOUD,
    ES_P_C_INFL, ES_P_DILUTION, ES_P_T_RATIO, ES_P_M_BD,
    ES_P_LOG_QC, ES_P_LOG_PC_BASE, ES_P_ALPHA_C, ES_P_LOG_R_EFF, ES_P_A_KH, ES_P_LOG_Q0, ES_P_F_CLD,
    ES_P_LOG_PC_TOP, ES_P_LOG_DPC, ES_P_FEAT_A, ES_P_FEAT_LAM0, ES_P_FEAT_W, ES_P_FEAT_XI,
    ES_P_N_EXTRA
};

#define ES_MAX_SPECIES 16
#define ES_MAX_LAYERS 112
#define ES_MAX_PARAMS (ES_MAX_SPECIES + ES_P_N_EXTRA)

/*
 * Static model description (Sect. 2.4 profile choice, Sect. 3 absorbers,
 * Sect. 4-5 geometry and star). Layers: n_layers (2..ES_MAX_LAYERS) with
 * n_layers+1 levels log-spaced from p_top (top) to p_bot (bottom); a
 * layer's pressure is the geometric mean of its levels. Hydrostatic
 * balance with g(r) = g_ref (R_p/r)^2 is anchored at r(p_ref) = R_p (the
 * derived R_bd with ES_FLUX_BROWN_DWARF).
 * theta_fixed holds every canonical slot's value; the user's parameter
 * vectors fill the n_free slots listed in free_idx (in that order).
 * Rayleigh cross-sections are sigma(nu) = ray_*_cm2 (nu / ray_nu_ref)^4.
 * emission_flux selects the emission output (ES_FLUX_*); distance_cm is
 * the brown dwarf's distance D (> 0 with ES_FLUX_BROWN_DWARF).
 * cloud_profile selects the non-grey cloud's q_c profile (ES_QC_*);
 * cloud_feature = 1 adds the mid-infrared feature to its Q_ext.
 * emission_quadrature selects the flux integral's angles (ES_QUAD_*).
 * emission_solver selects the emission RT (ES_RT_*); with ES_RT_DELTA_EAA,
 * cloud_ssa in [0, 1] and cloud_g in [0, 1) are the non-grey cloud's
 * single-scattering albedo and asymmetry parameter (constant in wavenumber;
 * the paper's cloud scheme gives Q_ext alone). These three trailing fields
 * are zero in a zero-initialised description: absorption-only emission.
 */
typedef struct {
    int n_layers;
    double p_top_bar, p_bot_bar, p_ref_bar;
    int tp_kind;                 /* ES_TP_*          */
    int cloud_kind;              /* ES_CLOUD_*       */
    int n_species;               /* S, 1..ES_MAX_SPECIES */
    double species_mass_amu[ES_MAX_SPECIES];
    double r_star_cm, t_star_k;
    double ray_h2_cm2, ray_he_cm2, ray_nu_ref;
    double theta_fixed[ES_MAX_PARAMS];
    int n_free;
    int free_idx[ES_MAX_PARAMS];
    int emission_flux;           /* ES_FLUX_*        */
    double distance_cm;
    int cloud_profile;           /* ES_QC_*          */
    int cloud_feature;           /* 0 or 1           */
    int emission_quadrature;     /* ES_QUAD_*        */
    int emission_solver;         /* ES_RT_*          */
    double cloud_ssa, cloud_g;   /* ES_RT_DELTA_EAA: cloud albedo, asymmetry */
} es_model_desc;

/*
 * Opacity tables (Sect. 3: opacity-sampled cross-sections on temperature
 * and pressure grids; H2-H2 and H2-He CIA). All host pointers, row-major:
 *   log10_sigma [n_species][n_t][n_p][n_nu]  log10 cm^2
 *   cia_h2h2, cia_h2he [n_t_cia][n_nu]        log10 cm^5
 * Grids strictly ascending; every species shares the wavenumber grid.
 * storage = ES_TABLE_BF16 keeps each (species, T, p) row as BF16 residuals
 * about an FP32 row offset (the row mean): value = bf16 + offset.
 */
typedef struct {
    int n_nu;      const double *nu;          /* cm^-1, ascending          */
    int n_t;       const double *t_grid;      /* K                          */
    int n_p;       const double *p_grid_bar;  /* bar                        */
    const float *log10_sigma;
    int n_t_cia;   const double *cia_t_grid;  /* K                          */
    const float *cia_h2h2;
    const float *cia_h2he;
    int storage;                              /* ES_TABLE_F32 | ES_TABLE_BF16 */
} es_tables_desc;

/* Create a context on CUDA device `device` for the model `desc`: the
 * pressure grid (Sect. 6.3: L layers evenly spaced in log p), the T-p profile
 * kind (Sect. 2.4), the absorbers (Sect. 3.1), the cloud scheme (Sect. 2.5),
 * the emission output and flux angles (Sect. 5). The context itself (a device
 * binding plus host state) has no counterpart in the paper.
 * Errors: ES_EINVAL (bad description), ES_ECUDA, ES_ENOMEM. */
es_status es_create(es_ctx **out, int device, const es_model_desc *desc);

/* Copy the opacity tables to the device (Sect. 3). Replaces earlier tables
 * and invalidates the instrument grid. Errors: ES_EINVAL (sizes, grids not
 * ascending, species count differs from the model), ES_ENOMEM, ES_ECUDA. */
es_status es_load_tables(es_ctx *ctx, const es_tables_desc *tables);

/* Instrument bins [lo, hi) in micron. The model of bin k is the equal-
 * weight mean of the native points with lambda = 1e4/nu in [lo_k, hi_k).
 * The paper compares binned data with the native-resolution model (Sect. 6-7)
 * but does not define the binning operator; this equal-weight mean is the
 * library's reading, not a passage of the paper.
 * Bins must not share native points; a bin with no points is ES_EINVAL.
 * Requires tables (ES_ESTATE). */
es_status es_set_grid(es_ctx *ctx, const double *bin_lo_um, const double *bin_hi_um, int n_bins);

/* Observed spectrum and 1-sigma errors for samples of `kind`
 * (transit depth for transmission, Fp/F* for emission), n_bins values
 * each, host memory (Sect. 2.3). Requires the grid (ES_ESTATE). */
es_status es_set_data(es_ctx *ctx, int kind, const double *y_obs, const double *sigma, int n_bins);

/* Set the batch: theta [batch][n_free] (the model's free slots, in
 * free_idx order) and kind [batch] (ES_KIND_*; NULL = all transmission),
 * both in `mem`: the parameter vectors a sampler proposes (Sect. 2.1-2.2; a
 * batch of live points per call is the library's addition). Grows the device
 * workspace as needed (ES_ENOMEM). */
es_status es_set_batch(es_ctx *ctx, const double *theta, const int32_t *kind, int batch,
                       int mem, es_stream_t stream);

/* Forward model for the current batch (Sects. 2.4-5) and its log-likelihood
 * (Sect. 2.3). Any output may be NULL:
 *   spectrum [batch][n_nu]  native-resolution transit depth or Fp/F* (float)
 *   binned   [batch][n_bins] binned model (double)
 *   lnL      [batch]          ln L (double); -1e300 for invalid samples
 * Needs tables, grid, data for every kind present, and a batch.
 * A batch of one transmission vector (the plain per-sample call) runs the
 * opacity stage (Sect. 3) as a kernel of its own: the raw table rows that
 * bracket the vector's layers, each read once, into the layer extinction,
 * which the chord kernel (Sect. 4) then reads (es_query key 17 gives the
 * row bytes); larger batches interpolate inside the fused kernels. With
 * ES_RT_DELTA_EAA the emission samples run through kernels of their own:
 * their extinction is stored per (sample, layer, wavenumber), then solved
 * column by column (the context holds that buffer and a scratch array). */
es_status es_forward(es_ctx *ctx, float *spectrum, double *binned, double *lnL,
                     int mem, es_stream_t stream);

/* ln L only (the sampler's call). Same requirements as es_forward.
 *
 * Bounded waits (es_forward, es_loglike, es_forward_backward): the
 * tensor-core kernels wait on mbarriers with an iteration limit. If one gives
 * up, every sample of the call gets ln L = -1e300, a zero gradient and the
 * flags ES_FLAG_INVALID | ES_FLAG_TIMEOUT; with host buffers (ES_MEM_HOST) the
 * call also returns ES_ETIMEOUT. The status is cleared at the start of every
 * call, so a later call that completes returns ES_OK. */
es_status es_loglike(es_ctx *ctx, double *lnL, int mem, es_stream_t stream);

/* ln L and its gradient with respect to the free parameters,
 * grad [batch][n_free] (double), by a hand-written adjoint that recomputes
 * the interpolated opacities (the paper motivates gradients through
 * automatic differentiation, Sect. 2.1, without computing them). Invalid samples get a zero gradient.
 * lnL or grad may be NULL (not copied out).
 *
 * CUDA-graph replay (es_loglike and es_forward_backward): the first call
 * after the batch shape, the tables, the grid or a buffer changed runs its
 * kernels directly; the next one captures the whole launch sequence into a
 * CUDA graph, and later calls replay it. Inputs and outputs go through the
 * context's own device buffers, so the graph stays valid when only theta
 * values (es_set_batch with the same batch and kind counts), data or output
 * pointers change. The graph runs on a private stream ordered after all
 * earlier work on `stream` by events, and later work on `stream` waits for
 * it. Disabled while profiling is on, or by es_set_graphs(ctx, 0). */
es_status es_forward_backward(es_ctx *ctx, double *lnL, double *grad, int mem,
                              es_stream_t stream);

/* Launch-shape autotuner of the fused persistent kernels (not a step of the
 * paper's method: tuning for this GPU). For the current batch's composition
 * (transmission only, emission only, or mixed: one kernel per direction over
 * both kinds) it times each kernel at several work-item sizes (wavenumber
 * tiles per item: 128-wavenumber tiles for transmission and mixed windows,
 * 512-wavenumber tiles for emission) and both work-item orders
 * (chunk-major: blocks running together share a wavenumber window of the
 * coefficient table in L2; sample-major: fewer sample stagings per block),
 * and keeps the fastest for later calls of this context (es_query keys 8, 9,
 * 12-16). Runs a full forward + adjoint plus a few dozen timed kernel
 * launches on `stream` and synchronises it; leaves the context's outputs
 * undefined until the next es_loglike / es_forward_backward. */
es_status es_autotune(es_ctx *ctx, es_stream_t stream);

/* CUDA-graph replay of es_loglike / es_forward_backward on (1, default) or
 * off (0). Either way drops any captured graph. No counterpart in the paper
 * (launch mechanics). */
es_status es_set_graphs(es_ctx *ctx, int on);

/* ln L of `batch` parameter vectors, like es_set_batch + es_loglike, but
 * without allocating any device memory: all per-call workspace comes from
 * one fixed array of 32 MiB built into the library (present on every GPU
 * that loads the library, until the process exits). The paper has no
 * counterpart; this is a library convenience for callers that must not call
 * cudaMalloc on their hot path (frameworks that own all device memory
 * through their own pool and forbid other allocations, or long runs that
 * must not risk an out-of-memory error mid-way).
 *   theta [batch][n_free] device, kind [batch] device or NULL (all
 *   transmission), lnL [batch] device; asynchronous on `stream`.
 * Needs tables, grid and transmission data (and emission data when kind is
 * given). kind values are not checked on the host (the call does not read
 * device memory back): a value other than ES_KIND_TRANSMISSION or
 * ES_KIND_EMISSION makes that sample invalid (ln L = -1e300). A kernel that
 * gives up on a bounded wait makes every ln L of the call -1e300.
 * A batch whose workspace exceeds 32 MiB is rejected with ES_EINVAL
 * (the message gives the bytes needed), and so is an emission batch (kind
 * given) of a model with ES_RT_DELTA_EAA, whose per-batch extinction buffer
 * does not fit the fixed array. The first call on a device looks up
 * the array's device address; make that first call before any stream
 * capture. All calls on a device share the array and leave their contents in
 * it: calls that overlap on the GPU race and must be serialised. */
es_status es_loglike_noalloc(es_ctx *ctx, const double *theta, const int32_t *kind, int batch, double *lnL,
                             es_stream_t stream);

/* Device memory limit of the context: `bytes` (0 = no limit, the default)
 * caps the device memory the context holds at any time (tables, grid, data,
 * workspace; es_query key 6). An allocation that would pass the limit fails
 * with ES_ENOMEM before anything is allocated, and the context keeps what it
 * held. No counterpart in the paper: sharing one GPU between contexts. */
es_status es_set_memory_limit(es_ctx *ctx, uint64_t bytes);

/* Test hooks, off (0) by default; no counterpart in the paper.
 * ES_TEST_WAIT_TIMEOUT: the tensor-core kernels issue no product and their
 * bounded waits give up after a few thousand polls (milliseconds), so the
 * next call takes its timeout path (ES_ETIMEOUT, ES_FLAG_TIMEOUT) with no
 * tensor-core operation in flight. Clearing it (hooks = 0) restores normal
 * calls on the same context. */
enum { ES_TEST_WAIT_TIMEOUT = 1 };
es_status es_set_test_hooks(es_ctx *ctx, int hooks);

/* Per-sample flags (ES_FLAG_*) of the last forward, int32 [batch]: which
 * samples got the paper's invalid-output ln L = -1e300 (Sect. 2.3), and why. */
es_status es_get_flags(es_ctx *ctx, int32_t *flags, int mem, es_stream_t stream);

/* Sizes and state of the context (no counterpart in the paper): 0 n_nu, 1 n_bins, 2 n_free, 3 batch, 4 n_layers, 5 n_species,
 * 6 device bytes the context holds, 7 kernel launches issued by the last call (a
 * replayed graph counts the launches it holds), 8 / 9 work-item size of the
 * fused transmission forward / adjoint kernel (0: built-in heuristic),
 * 10 graph replay enabled (1) or not (0), 11 device status word of the last
 * call (0; nonzero when a tensor-core kernel gave up on a bounded wait;
 * synchronises), 12 / 13 work-item size of the fused emission forward /
 * adjoint (512-wavenumber tiles), 14 / 15 window of the mixed forward /
 * adjoint (128-wavenumber tiles), 16 work-item orders (bit k set: kernel k
 * of trans fwd, trans bwd, emis fwd, emis bwd, mixed fwd, mixed bwd runs its
 * items sample-major). Sizes 0: the built-in heuristic.
 * 17 bytes of raw table rows and CIA rows the one-vector opacity stage read
 * for the last call (the union of the rows bracketing the vector's layers,
 * over all wavenumbers; 0 when the last call did not run that stage;
 * synchronises).
 * Returns -1 for an unknown key or a NULL context. */
int64_t es_query(const es_ctx *ctx, int key);

/* Per-kernel timing with CUDA events recorded on the launching stream
 * around every kernel launch of later calls (on = 1) or off (on = 0, the
 * default). Turning it on or off clears the accumulated times. No
 * counterpart in the paper (measurement). */
es_status es_set_profiling(es_ctx *ctx, int on);

/* Accumulated profile entry `index` (0-based, in first-launch order; no
 * counterpart in the paper):
 * copies the kernel's name (NUL-terminated, at most name_len bytes), its
 * total device time in milliseconds and its launch count. Synchronises the
 * device. Returns ES_EINVAL when index is past the last entry. */
es_status es_get_profile(es_ctx *ctx, int index, char *name, int name_len, double *total_ms,
                         int64_t *launches);

/* Throughput probe of GPU `device` (not a step of the paper's method; a
 * measured ceiling for the ALU roofline of the interpolation kernels):
 * ex2.approx.ftz.f32 instructions per second and packed FP32x2 FMA
 * instructions per second, each from a kernel of independent dependency
 * chains at full occupancy (best of three ~ms runs). Synchronous; allocates
 * and frees 1 KB. ES_EINVAL for NULL outputs, ES_ECUDA for a bad device. */
es_status es_probe_rates(int device, double *ex2_per_s, double *ffma2_per_s);

/* Message for the last error on this context (never NULL). Library
 * plumbing with no counterpart in the paper. */
const char *es_last_error(const es_ctx *ctx);

/* Free every device and host resource of the context. NULL is a no-op.
 * Library plumbing with no counterpart in the paper. */
void es_destroy(es_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* EXOSKRY_H */
