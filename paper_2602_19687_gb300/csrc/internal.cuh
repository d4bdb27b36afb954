// Internal declarations shared by the C-ABI layer and the kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "exoskry.h"

namespace es {

// CODATA 2018 (cgs) and nominal radii
constexpr double K_B = 1.380649e-16;
constexpr double H_PLANCK = 6.62607015e-27;
constexpr double C_LIGHT = 2.99792458e10;
constexpr double AMU = 1.66053906660e-24;
constexpr double R_JUP = 7.1492e9;
constexpr double BAR = 1.0e6;
constexpr double PI = 3.14159265358979323846;
constexpr double LN10 = 2.302585092994045684;
constexpr double LOG2_10 = 3.321928094887362348;
// Sect. 3.1 background gas; Sect. 2.4.4 modified Guillot constants
constexpr double HE_TO_H2 = 0.164;
constexpr double M_H2 = 2.01588;
constexpr double M_HE = 4.002602;
constexpr double F_HEM = 0.25;
constexpr double Q_INT = 2.0 / 3.0;
constexpr double Q_IRR_INF = 2.0 / 3.0;
// Sect. 2.4.3 modified Milne: q_inf fixed at the grey Hopf function's deep
// limit q(infinity) (the paper quotes it as ~0.71)
constexpr double Q_MILNE_INF = 0.7104460895;
// Sect. 5 brown dwarfs: R_bd = sqrt(G M_bd / g); CODATA 2018 G, nominal Jupiter mass
constexpr double G_GRAV = 6.67430e-8;
constexpr double M_JUP = 1.89813e30;
// Sect. 2.3: invalid forward-model output
constexpr double INVALID_LNL = -1.0e300;
// second radiation constant h c / k_B [cm K] and 2 h c^2 [erg cm^2 s^-1]
constexpr double C2_RAD = H_PLANCK * C_LIGHT / K_B;
constexpr double TWO_HC2 = 2.0 * H_PLANCK * C_LIGHT * C_LIGHT;
// Species slots per lane in the fused transmission kernels (two lanes share a
// wavenumber pair and split the species between them).
__host__ __device__ constexpr int spl_for(int S) { return S <= 4 ? 2 : (S <= 8 ? 4 : 8); }
// number of Gauss-Legendre angles for the emission flux integral
// per-sample constants of the non-grey cloud's g(nu) = Q_ext / Q_1 and the
// slots of their adjoints: (2 pi r_eff | ln r_eff, a, Q0 | ln Q0, f_cld, A,
// lambda_0, omega, xi)
constexpr int N_CG = 8;
constexpr int N_MU = 4;
// reductions per (sample, layer) in the extinction adjoint, each a sum over
// wavenumber of alpha_bar times a part of d alpha: 0/1 QS (species sum; two
// partial sums added by the reader), 2/3 D (temperature slope of the species
// sum; two partials), 4 C1, 5 C2 (CIA terms), 6 C1T, 7 C2T (their temperature
// slopes), 8 W4 (Rayleigh weight). Per-species totals over layers go to
// Work::qtot; for transmission, W4 comes from Work::zbar instead of slot 8.
constexpr int N_RED = 9;

// Constant model data, passed by value to every kernel.
struct Model {
    int L, S, NT, NP, NTc, N, nbins, nfree, nfull;
    int Np;                       // padded row stride of tables and per-wavenumber arrays (N rounded up to 128)
    int SP;                       // species slots per coefficient-table entry (2 spl_for(S) >= S)
    int tp_kind, cloud_kind, bf16;
    int cloud_profile;            // ES_QC_* (non-grey cloud)
    int cloud_feature;            // 1: the mid-infrared feature in Q_ext
    int emis_flux;                // ES_FLUX_*
    // bounded mbarrier waits of the tensor-core kernels: polls before giving
    // up; wait_test = 1 (es_set_test_hooks) also skips issuing their products,
    // so that every wait runs out with no tensor-core operation in flight
    unsigned wait_polls;
    int wait_test;
    double distance;              // cm (brown-dwarf flux)
    double p_ref;                 // dyn cm^-2
    double r_star, t_star;
    double ray_h2, ray_he, ray_nu_ref;
    double mass[ES_MAX_SPECIES];
    int free_idx[ES_MAX_PARAMS];
    double theta_fixed[ES_MAX_PARAMS];
    double mu_gl[N_MU], w_gl[N_MU];   // flux angles mu_j and weights w_j (F = 2 pi sum w_j mu_j I_j)
    // emission solver (ES_RT_*); the delta-EAA's interpolatory weights of
    // int_0^1 dmu at the flux angles, and the cloud's albedo and asymmetry
    int emis_solver;
    double c_mu[N_MU];
    float cloud_ssa, cloud_gasym;
    // device arrays
    const double *p_lev, *p_lay;  // [L+1], [L]
    const double *lnp_lev;        // [L+1] ln p_lev
    double ln_p_ref;              // ln p_ref
    const int *ip;                // [L] pressure bracket of each layer
    const float *wp;              // [L] pressure weight of each layer
    const double *log_t;          // [NT] log10 of the temperature grid
    const double *cia_t;          // [NTc]
    const float *tab32;           // [S][NT][NP][Np]
    const uint16_t *tab16;        // [S][NT][NP][Np] BF16 residuals
    const float *row_off;         // [S][NT][NP] (zeros for FP32 tables)
    const float4 *coef4;          // [(NT-1)(NP-1) cells][SP/2 j][2 c][Np/2 pairs][2 h] bilinear coefficients
                                  // (log2 units) (v00, v01 - v00, v10 - v00, v11 - v10 - v01 + v00) x log2(10)
                                  // of species slot s = h SP/2 + j: c = 0 (c0, c0', c1, c1'), c = 1
                                  // (c2, c2', c3, c3') for a wavenumber pair; slots >= S zero
    const float4 *cia4;           // [NTc-1][Np/2 pairs][2 CIA pairs] (b, b', d, d'): b = log2(10) log10 k(T_i),
                                  // d = log2(10) (log10 k(T_i+1) - log10 k(T_i))
    const float *cia;             // [2][NTc][Np] log10 k
    const float *nu;              // [Np]
    const float *inv_fstar;       // [Np] 1 / (pi B(T_*, nu))
    const int *bin_lo, *bin_hi;   // [nbins] native index ranges [lo, hi)
    const int *bin_of;            // [N] bin of each native point or -1
    const double *y_obs, *sigma;  // [2][nbins]
};

// Per-batch device workspace.
struct Work {
    int B;
    const double *theta_user;     // [B][nfree]
    double *theta;                // [B][nfull]
    int *kind, *flags;            // [B]
    int *err;                     // [1] nonzero once a kernel gave up on a bounded wait (cleared per call)
    double *t_lay, *t_lev, *r_lev;// [B][L], [B][L+1], [B][L+1]
    double *xs;                   // [B][S+2] X_s..., X_H2, X_He
    double *n_lay;                // [B][L]
    double *rc, *base, *scale;    // [B]
    float *lmat;                  // [B][L][L] path lengths L_il = P_il dr_l
    float *area;                  // [B][L] annulus area / R_*^2
    float *dr;                    // [B][L]
    int *it;                      // [B][L] temperature bracket
    float *gt;                    // [B][L] 1/dlog10T of the bracket (0 if clamped)
    float *wtr;                   // [B][L] raw temperature weight
    int *itc;                     // [B][L] CIA temperature bracket
    float *wtc, *gtc;             // [B][L] CIA weight, 1/dT (0 if clamped)
    float *ccia;                  // [B][L][2] log2(n^2 X_H2 X_H2), log2(n^2 X_H2 X_He)
    float *ray;                   // [B][L] n (X_H2 s_H2 + X_He s_He)
    // non-grey cloud (ES_CLOUD_KH18): extinction C_l g(nu), g = 1/(Q0 x^-a + x^0.2)
    float *cloud_c;               // [B][L] C_l = 3 rho_a q_c^eff / (4 r_eff)
    float *cloud_d;               // [B][L] D_i = sum_l L_il C_l: cloudy chord depth = tau_i + g(nu) D_i
    float *cloud_g;               // [B][N_CG] 2 pi r_eff [cm], a, Q0, f_cld, A (0: no feature), lambda_0, omega, xi
    float *spec;                  // [B][N] transmission: depth - base; emission: Fp/F*
    // one-vector transmission path: the extinction of the opacity stage, and
    // per sample the table rows (species x nodes) and CIA rows it read
    float *ext;                   // [B][L][Np]
    int *arows;                   // [B][2]
    double *ymod;                 // [B][nbins]
    double *lnl;                  // [B]
    // adjoint
    float *dbar;                  // [B][Np] d lnL / d spec (zero beyond N)
    float *estore;                // [B][L][Np] exp(-tau) of the forward (transmission adjoint)
    float *lbar;                  // [B][L][L] (FP32 atomics: one partial per work item)
    double *red;                  // [B][L][N_RED]
    double *qtot;                 // [B][S] per-species reductions summed over layers
    double *zbar;                 // [B][L] transmission: sum_nu tau_bar_i(nu) (nu/nu_ref)^4
    float *itop;                  // [B][Np][1 or 2][4] emission: top-of-atmosphere intensity per angle of the
                                  // clear (and, with the non-grey cloud, the cloudy) column, for the adjoint
    double *areabar;              // [B][L]
    double *levbar;               // [B][L+1] d lnL / d T_lev (emission)
    double *drbar;                // [B][L]   d lnL / d dr (emission)
    double *misc;                 // [B][4] base_bar, scale_bar, c_bar, -
    double *cloud_dbar;           // [B][L] non-grey cloud: d lnL / d D_i (transmission), d lnL / d C_l (emission)
    double *cloud_pbar;           // [B][N_CG] d lnL / d (ln r_eff via g, a, ln Q0, f_cld, A, lambda_0, omega, xi)
    double *grad;                 // [B][nfree]
};

// Optional per-launch callbacks (CUDA-event profiling of each kernel).
struct Hook {
    void *ctx = nullptr;
    void (*begin)(void *, const char *, cudaStream_t) = nullptr;
    void (*end)(void *, cudaStream_t) = nullptr;
    void on_begin(const char *name, cudaStream_t s) const { if (begin) begin(ctx, name, s); }
    void on_end(cudaStream_t s) const { if (end) end(ctx, s); }
};
#define ES_LAUNCH(hook, name, st, ...) \
    do {                                 \
        (hook).on_begin(name, st);       \
        __VA_ARGS__;                     \
        (hook).on_end(st);               \
    } while (0)

// kernel launchers (each returns the number of kernels launched)
int launch_build_coef(const Model &m, float4 *coef, cudaStream_t st);
int launch_setup(const Model &m, const Work &w, cudaStream_t st, const Hook &h);
// Fused persistent kernels. chunk: wavenumber tiles per work item (<= 0:
// built-in heuristic); sample_major: work-item order (0 chunk-major, 1
// sample-major). Transmission tiles are 128 wavenumbers, emission tiles 512;
// the mixed kernels' window `wtiles` counts 128-wavenumber tiles (rounded to
// whole emission tiles).
// fused emission: interpolation + Schwarzschild integration (store_i keeps I_toa for the adjoint)
int launch_emis_fused_forward(const Model &m, const Work &w, bool store_i, int chunk, int sample_major,
                              cudaStream_t st, const Hook &h);
// delta-EAA emission with scattering (k_eaa.cu): the extinction store and the
// RT kernel; the RT adjoint and the interpolation adjoint. scr: a scratch
// array of eaa_scratch_floats(m) floats.
size_t eaa_scratch_floats(const Model &m);
int launch_eaa_forward(const Model &m, const Work &w, float *scr, bool store_i, cudaStream_t st, const Hook &h);
int launch_eaa_backward(const Model &m, const Work &w, float *scr, cudaStream_t st, const Hook &h);
int launch_emis_fused_backward(const Model &m, const Work &w, int chunk, int sample_major, cudaStream_t st,
                               const Hook &h);
int launch_trans_fused_forward(const Model &m, const Work &w, bool store_e, int chunk, int sample_major,
                               cudaStream_t st, const Hook &h);
int launch_trans_fused_backward(const Model &m, const Work &w, int chunk, int sample_major, cudaStream_t st,
                                const Hook &h);
// one kernel per direction over both kinds of a mixed batch (store: exp(-tau) and I_toa for the adjoint)
int launch_mixed_fused_forward(const Model &m, const Work &w, bool store, int wtiles, int sample_major,
                               cudaStream_t st, const Hook &h);
int launch_mixed_fused_backward(const Model &m, const Work &w, int wtiles, int sample_major, cudaStream_t st,
                                const Hook &h);
// One-vector transmission path: the opacity stage (extinction of every layer
// and wavenumber from the raw table rows into w.ext) and the chord kernel
// that reads it (transit depth; store_e keeps exp(-tau) for the adjoint)
int launch_trans_alpha(const Model &m, const Work &w, cudaStream_t st, const Hook &h);
int launch_trans_chord_forward(const Model &m, const Work &w, bool store_e, cudaStream_t st, const Hook &h);
// tiles per work item of the transmission kernels' heuristic
int chunk_tiles(const Model &m, int B, int blocks, int tile);
int launch_bins(const Model &m, const Work &w, bool want_adjoint, float *spectrum_out,
                double *binned_out, double *lnl_out, cudaStream_t st, const Hook &h);
// lnl_out: the call's ln L output, set to -1e300 for every sample when a kernel gave up on a bounded wait
int launch_setup_backward(const Model &m, const Work &w, double *lnl_out, cudaStream_t st, const Hook &h);

}  // namespace es
