// hr2_internal.cuh -- device-side data structures shared by the kernels and
// the host implementation of the C ABI (include/hr2.h).
#pragma once
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "hr2.h"

namespace hr2 {

// Wavenumber tile of one work item: 32 lanes x 2 packed pairs of
// consecutive points (lane l holds columns 2l, 2l+1, 64+2l, 65+2l).
constexpr int kTileNu = 128;
// distance in points between a lane's consecutive packed pairs
constexpr int kPairStride = 64;
constexpr int kMaxWarps = 16;
// launch bounds of the FP32 forward kernel: at most 4 warps (samples) per
// CTA.  The level-gridded linear-source kernels with up to 4 angle nodes are
// budgeted for 4 resident CTAs of 4 warps (16 warps per SM, 128 registers);
// the others (more nodes, the parabolic source, the direct path) for 3
// (12 warps, 170 registers).
constexpr int kForwardMaxThreads = 128;
constexpr int kForwardMinBlocks = 3;
constexpr int kForwardMinBlocksSmall = 4;
// shared-memory stages per warp of the level-gridded forward kernel, for a
// kernel with nmu angle nodes, compiled absorber bound kt (0: runtime count)
// and a batch of n samples.  One stage (more warps per SM fit; each level's
// copy lands while its source and layer run) for the linear-source kernels
// with up to 4 nodes, and for those with a bound of 8 or more on batches of at
// least kOneStageMinBatch samples; two (the copy is issued a whole level
// ahead, which few warps per SM need to hide its latency) otherwise.  The
// kernels exist in exactly these variants.
constexpr int kOneStageMinBatch = 16;
__host__ __device__ constexpr int forward32_stages(int nmu, bool para, int kt, int n) {
  return (para || kt == 0) ? 2 : (nmu <= 4 ? 1 : ((kt >= 8 && n >= kOneStageMinBatch) ? 1 : 2));
}
// whether that kernel exists with one and with two stages (a launch shape may
// then ask for either)
__host__ __device__ constexpr bool forward32_has_both_depths(int nmu, bool para, int kt) {
  return !para && kt >= 8 && nmu > 4;
}// dynamic shared memory the cached forward kernel may use per CTA
constexpr size_t kForwardSmemCap = 200u * 1024u;
constexpr int kCiaH2H2 = HR2_MAX_SPECIES;      // offset slot of the H2-H2 CIA table
constexpr int kCiaH2He = HR2_MAX_SPECIES + 1;  // offset slot of the H2-He CIA table

// Bounds-checked build (compiled with -DHR2_BOUNDS_CHECK=1; a debugging aid
// in place of a device memory checker): index checks ahead of the accesses
// they guard.  A failed check sets bit 1 of the batch's error word (the host
// reports HR2_EBOUNDS) and the guarded work is skipped, so nothing reads or
// writes outside its buffer.  In the normal build the checks compile to
// nothing.
#ifndef HR2_BOUNDS_CHECK
#define HR2_BOUNDS_CHECK 0
#endif
constexpr int kErrWait = 1;     // error-word bit: a bounded wait gave up
constexpr int kErrBounds = 2;   // error-word bit: an index check failed (bounds-checked build)
__device__ __forceinline__ bool bounds_ok(bool ok, int* err) {
#if HR2_BOUNDS_CHECK
  if (!ok && err) atomicOr(err, kErrBounds);
  return ok;
#else
  (void)err;
  return ok || true;
#endif
}

// CGS constants (CODATA 2018).
constexpr double kH = 6.62607015e-27;         // erg s
constexpr double kC = 2.99792458e10;          // cm s^-1
constexpr double kKB = 1.380649e-16;          // erg K^-1
constexpr double kAMU = 1.66053906660e-24;    // g
constexpr double kParsec = 3.0856775814913673e18;  // cm
constexpr double kBar = 1.0e6;                // dyn cm^-2
constexpr double kMassH2 = 2.01588;           // u
constexpr double kMassHe = 4.002602;          // u
constexpr double kPi = 3.141592653589793;
constexpr double kLog2_10 = 3.321928094887362;    // log2(10)
constexpr double kLog2e = 1.4426950408889634;     // log2(e)
constexpr double kLn2 = 0.6931471805599453;       // ln(2)
// second radiation constant h c / k_B (cm K) and 2 h c^2 (erg cm^2 s^-1)
constexpr double kC2 = kH * kC / kKB;
constexpr double kC1 = 2.0 * kH * kC * kC;
// Stefan-Boltzmann constant 2 pi^5 k^4 / (15 h^3 c^2), erg s^-1 cm^-2 K^-4
constexpr double kSigmaSB = 2.0 * kPi * kPi * kPi * kPi * kPi * kKB * kKB * kKB * kKB / (15.0 * kH * kH * kH * kC * kC);

// Hopf function table of Milne's profile: q at ln tau uniform on
// [ln kHopfTau0, ln kHopfTau1] (kHopfN points); q(0) below, q(kHopfTau1)
// above (q approaches q(inf) within e^-60 there)
constexpr int kHopfN = 4096;
constexpr double kHopfTau0 = 1e-9;
constexpr double kHopfTau1 = 60.0;

// Device copy of one opacity table set.
struct TablesDev {
  int storage;            // HR2_STORE_*
  int n_species, n_T, n_p, n_nu, nu_pad;
  double nu0, dnu;
  const __half* sig16;    // [n_species][n_T][n_p][nu_pad]  (FP16 of value - off_s)
  const __half* cia16;    // [2][n_T][nu_pad] (H2-H2, H2-He) or null
  const double* sig64;    // [n_species][n_T][n_p][nu_pad]
  const double* cia64;    // [2][n_T][nu_pad] or null
  int has_cia[2];
  // FP16 offsets off_s: [0, HR2_MAX_SPECIES) species, then kCiaH2H2, kCiaH2He
  double off[HR2_MAX_SPECIES + 2];
  float T_grid[HR2_MAX_TGRID];
  double T_grid64[HR2_MAX_TGRID];
  double log10p_grid64[HR2_MAX_PGRID];
  double mass[HR2_MAX_SPECIES];
};

// Per-level data of a setup that does not depend on the sample.
struct LevelDev {
  int pcell;              // p-grid cell index b_j (clamped)
  float wp;               // weight of log10p_grid[b_j + 1]
  float p_dyn;            // level pressure, dyn cm^-2
  float half_dp;          // (p_{j+1} - p_j) / 2 for layer j (0 for the last level)
  double p_dyn64, half_dp64;
  double wp64;
  double lpk;             // log2(p_j / k_B): the level's part of log2 n_j = lpk - log2 T_j
};

// Device descriptor of one setup (lives in device memory).
struct SetupDev {
  int nu_first, n_nu;     // table columns used
  int tile0, n_tiles;     // kTileNu-aligned tiles (in table columns) covering the range
  int n_lev;              // levels = layers + 1
  int n_species;
  int species[HR2_MAX_SPECIES];
  float mass[HR2_MAX_SPECIES];
  double mass64[HR2_MAX_SPECIES];
  int n_mu;
  float mu_nlog2e[HR2_MAX_MU];   // -log2(e) / mu_k
  float mu[HR2_MAX_MU];
  float inv_mu[HR2_MAX_MU];
  float wflux[HR2_MAX_MU];       // 2 pi w_k mu_k
  // log2(2 pi w_k mu_k^2): the node's share of F+ = sum_k 2 pi w_k mu_k^2
  // (I_0(mu_k) / mu_k), folded into its transmission exponential (-1e4 for a
  // padded node of zero weight)
  float lwmu[HR2_MAX_MU];
  double mu64[HR2_MAX_MU], wmu64[HR2_MAX_MU];  // Gauss-Legendre nodes and weights on [0,1]
  int fe_elements, fe_order, n_tnodes;
  double gll[HR2_MAX_TNODES];    // Gauss-Lobatto nodes on [0,1] (fe_order+1 of them)
  // finite-element profile at the levels (set up once): element of level j
  // and the values of its fe_order+1 Lagrange basis functions there
  const int* fe_k;               // [n_lev]
  const double* fe_b;            // [n_lev][fe_order + 1]
  double r_he, radius_cm;
  int n_bins;
  long long w_nnz;
  const LevelDev* levels;        // [n_lev]
  const long long* w_rowptr;     // [n_bins+1]
  const int* w_col0;             // [n_bins] first setup point of row b
  const float* w32;              // [nnz]
  const double* w64;             // [nnz]
  const double* obs_D;           // [n_bins] or null
  const double* obs_sigma;       // [n_bins] or null
  // with the observation (k_obs_terms): 1 / (2 sigma_b^2) per bin and
  // sum_b -ln(2 pi sigma_b^2) / 2, the likelihood's terms that do not depend
  // on the model when there is no error inflation
  const double* obs_inv2s2;      // [n_bins] or null
  const double* obs_lnorm;       // [1] or null
  float cost;                    // relative cost of one work item (scheduling)
  const TablesDev* tables;       // device copy
  // level-gridded operand (level_cache): the tables interpolated in p onto
  // the levels, FP32, columns local to the setup's tiles
  int cached;
  // per T cell a: the row of T row a and the difference to row a+1,
  // interleaved per pair of columns ({g[2q], g[2q+1], dg[2q], dg[2q+1]}),
  // for the absorbers and then the two CIA pairs
  const float* lvl32;            // [n_tiles][n_lev][n_T - 1][n_species + 2][kTileNu / 2][4]
  long long lvl32_tile_floats;   // floats of one tile of that operand
  // wavenumber constants of the FP32 kernel per pair q of setup-local
  // columns 2q, 2q+1 (tile t holds pairs t kTileNu/2 ...): the first point's
  // wavenumber as an FP32 head and tail, nu_{2q+1} / nu_{2q}, and c1 nu^3 of
  // both points (FP64 arithmetic at creation)
  const float4* nu_pair;         // [n_tiles * kTileNu / 2] {head, tail, ratio, 0}
  const float2* c1n_pair;        // [n_tiles * kTileNu / 2]
  // temperature profile (HR2_PROFILE_*); Milne's profile reads its Hopf
  // function from hopf_q [kHopfN] (built at setup creation)
  int profile;
  const double* hopf_q;
  int cloud;                     // gray cloud layer from parameters HR2_P_CLOUD..
  int sc;                        // HR2_SC_LINEAR or HR2_SC_PARABOLIC source interpolation
  // interpolation space (HR2_INTERP_*): with HR2_INTERP_LINEAR the operand
  // holds 10^(stored log10 sigma) interpolated linearly in log10 p (and the
  // CIA operand 10^(stored value)), and the kernels interpolate linearly in T
  int interp;
};

// Per-(sample, level) inputs of the FP32 forward kernel, written by the
// prep kernel: table row, interpolation weights, CIA terms and Planck
// factors.  Four 16-byte words.
//
// Exponents are kept small and exact in FP32: every exponent of the sample
// is shifted by an integer power of two 2^shift (undone exactly in half_dp),
// and each per-sample constant is split into an FP32 head and a tail that
// enters as the factor (1 + ln2 * tail) on the exponential.
struct __align__(16) LevRec {
  int rowoff;        // a_j * n_p + b_j: row of corner (T cell a_j, p cell b_j)
  float wT;          // weight of T_grid[a_j + 1]
  float wp;          // weight of log10p_grid[b_j + 1]
  float wTwp;        // wT * wp
  float bh2h2;       // head of log2(x_H2^2 c n_j) + off_cia log2(10) - shift
  float bh2he;       // head of log2(x_H2 x_He c n_j) + off_cia log2(10) - shift
  float upl;         // log2(e) h c / (k T_j): e^{hc nu/kT} = 2^(upl nu)
  float half_dp;     // 2^shift (p_{j+1} - p_j) / 2, dyn cm^-2 (layer j)
  int acell;         // a_j
  float r64;         // e^{64 h c dnu / (k T_j)}: Planck factor between points 64 apart
  float ch2h2;       // 1 + ln2 * (tail of bh2h2)
  float ch2he;       // 1 + ln2 * (tail of bh2he)
  float rnu;         // e^{h c dnu / (k T_j)}: Planck factor between neighbouring points
  float wh2h2;       // 2^(bh2h2 exactly): the H2-H2 factor as a weight
  float wh2he;       // 2^(bh2he exactly)
  float dtau_cloud;  // gray cloud optical depth of layer j-1 (between levels j-1 and j),
                     // + kTinyTau on the linear-source path
};

// The same record as the level-gridded (cached) sweep reads it: the factors
// it applies to packed pairs of wavenumbers are stored twice, so that they
// load straight into register pairs.  Written instead of LevRec for setups
// with the level-gridded operand (a batch holds setups of one kind).
struct __align__(16) LevRecC {
  float wT[2];       // weight of T_grid[a_j + 1]
  float wh2h2[2];    // H2-H2 factor as a weight (0 for an absent pair)
  float wh2he[2];    // H2-He factor as a weight (0 for an absent pair)
  float half_dp[2];  // 2^shift (p_{j+1} - p_j) / 2, dyn cm^-2 (layer j)
  float dtc[2];      // gray cloud optical depth of layer j-1 (+ kTinyTau, linear source)
  float upl;         // log2(e) h c / (k T_j): e^{hc nu/kT} = 2^(upl nu)
  float rnu;         // e^{h c dnu / (k T_j)}
  int acell;         // a_j
  int lvl_off;       // floats from a tile's operand to this level's block of T cell a_j
  float r64;         // e^{64 h c dnu / (k T_j)}
  int pad;
};
static_assert(sizeof(LevRecC) == sizeof(LevRec), "both level records are 64 bytes");
constexpr int kRecCAcell = 12;   // float index of LevRecC::acell (lvl_off follows)
constexpr int kRecCUpl = 10;     // float index of LevRecC::upl

// Per-sample scalars written by the prep kernel.
struct SampleDev {
  float A[HR2_MAX_SPECIES];   // head of log2(x_s c) + off_s log2(10) - shift, c = 1/(mmw m_u g)
  float Ac[HR2_MAX_SPECIES];  // 1 + ln2 * (its tail)
  float W[HR2_MAX_SPECIES];   // 2^(log2(x_s c) + off_s log2(10) - shift): the same factor as a weight
  double scale;               // f (R_* / d)^2
  float scale32[2];           // the same as an FP32 head and tail
  int status;                 // HR2_SAMPLE_* bits
  int setup;                  // setup index, -1 if invalid
};

// Work plan written by the planner kernel for one batch call.
struct PlanDev {
  int total_items;
  int n_setups;
  int order[HR2_MAX_SETUPS];        // setups in decreasing item cost
  int count[HR2_MAX_SETUPS];        // samples per setup
  int first[HR2_MAX_SETUPS];        // start of the setup's samples in perm
  int n_sblocks[HR2_MAX_SETUPS];    // sample blocks per setup
  int item_start[HR2_MAX_SETUPS + 1];  // by position in `order`
};

struct FwdArgs {
  const SetupDev* setups[HR2_MAX_SETUPS];
  int n_setups;
  int n;
  const int* setup_of_sample;
  const double* params;
  const int* perm;          // samples grouped by setup
  const PlanDev* plan;
  unsigned int* counter;    // work counter (reset by the planner)
  float* highres;           // [n][highres_ld]: F+ (caller's or workspace)
  int highres_ld;
  double* highres64;        // FP64 path: F+ [n][highres64_ld] in the workspace
  int highres64_ld;
  float* user_highres;      // FP64 path: optional FP32 copy for the caller
  int* status;              // [n] or null
  LevRec* recs;             // [n][rec_ld]
  int rec_ld;
  SampleDev* samp;          // [n]
  int warps;                // samples per work item
  int tiles_per_item;       // consecutive kTileNu-point tiles per work item
  int* err;                 // device error word (bit 0: a bounded wait gave up), or null
  long long wait_limit;     // SM clock cycles a pipeline wait may take before it gives up
  unsigned tx_extra;        // test hook: bytes each item's first stage waits for in vain (0)
  // angle-node constants of the linear-source sweep per setup g and node k,
  // each as a pair of equal floats (one packed operand): 1/mu_k and
  // log2(2 pi w_k mu_k^2); kernel parameters, so that the sweep reads them
  // through the constant cache instead of shared memory
  unsigned long long node_im[HR2_MAX_SETUPS][HR2_MAX_MU];
  unsigned long long node_lw[HR2_MAX_SETUPS][HR2_MAX_MU];
  // the parabolic-source sweep's other two node constants of setup 0,
  // -log2(e)/mu_k and mu_k, for launches with a single setup (the general
  // sweep reads all three from shared memory)
  unsigned long long node_mnl0[HR2_MAX_MU];
  unsigned long long node_mu0[HR2_MAX_MU];
  // two-pass direct path (small batches on FP16 tables without the operand):
  // absorption coefficients [n][rec_ld levels][chi_ld setup-local columns],
  // written by k_chi_direct and read by the sweep; null otherwise
  float* chi;
  long long chi_ld;
};
// default of the context's wait limit: ~1 s of SM clock
constexpr long long kDefaultWaitCycles = 2000000000ll;
// default of the largest batch the direct path evaluates in two passes
constexpr int kDefaultSplitMaxBatch = 2;

// Launchers (kern_*.cu).
cudaError_t launch_prep(const FwdArgs& a, cudaStream_t s);
cudaError_t launch_plan(const FwdArgs& a, int* perm, PlanDev* plan, cudaStream_t s);
// kt: 0, or an even bound on the absorber count of the cached path with
// every setup of the batch at kt or kt - 1 absorbers (see absorber_bound)
cudaError_t launch_forward32(const FwdArgs& a, int max_nmu, int grid, bool cached, bool linear, bool para, int max_k,
                             int kt, int stages, cudaStream_t s);
// the same for one angle-node count (kern_fwd32_inst.cu)
#define HR2_DECLARE_FWD32(N)                                                                                 \
  cudaError_t launch_forward32_n##N(const FwdArgs& a, int grid, bool cached, bool linear, bool para, int max_k, \
                                    int kt, int stages, cudaStream_t s);
HR2_DECLARE_FWD32(1)
HR2_DECLARE_FWD32(2)
HR2_DECLARE_FWD32(3)
HR2_DECLARE_FWD32(4)
HR2_DECLARE_FWD32(5)
HR2_DECLARE_FWD32(6)
HR2_DECLARE_FWD32(7)
HR2_DECLARE_FWD32(8)
#undef HR2_DECLARE_FWD32
size_t forward32_smem_bytes(int warps, int max_k, int stages);
cudaError_t launch_forward64(const FwdArgs& a, int max_nmu, int max_nu, cudaStream_t s);
cudaError_t launch_bins(const FwdArgs& a, float* bins, int bins_ld, bool fp64, cudaStream_t s);
// first pass of the two-pass direct path: chi of every (sample, level, tile)
cudaError_t launch_chi_direct(const FwdArgs& a, int max_lev, int max_tiles, cudaStream_t s);
struct LnlArgs {
  const SetupDev* setups[HR2_MAX_SETUPS];
  int n_setups;
  const int* setup_of_sample;
  const float* bins;
  int bins_ld;
  const double* log_eps;
  int n;
  double* lnl;
};
cudaError_t launch_lnl(const LnlArgs& a, cudaStream_t s);
cudaError_t launch_obs_terms(const double* sigma, int n_bins, double* inv2s2, double* lnorm, cudaStream_t s);
// Hopf function table (kern_setup.cu) and effective temperatures (kern_forward.cu)
cudaError_t build_hopf_table(double* d_q, cudaStream_t s);
cudaError_t build_fe_basis(int n_lev, int fe_elements, int fe_order, const double* gll, int* d_k, double* d_b,
                           cudaStream_t s);
cudaError_t launch_teff(const FwdArgs& a, const float* highres, int highres_ld, double* out, cudaStream_t s);
// nested-sampling evidence bookkeeping (kern_nested.cu)
cudaError_t launch_ns_init(hr2_ns_state* st, cudaStream_t s);
cudaError_t launch_ns_propose(int n_live, const double* live_theta, const double* lo, const double* hi,
                              double enlarge, int n, double* box, double* out, unsigned long long seed,
                              unsigned long long counter, cudaStream_t s);
cudaError_t launch_ns_absorb(int n_live, double* live_lnl, double* live_theta, int n_cand, const double* cand_lnl,
                             const double* cand_theta, hr2_ns_state* st, double* dead_lnl, double* dead_logw,
                             double* dead_theta, long long dead_cap, cudaStream_t s);
cudaError_t launch_ns_finalize(int n_live, const double* live_lnl, const hr2_ns_state* st, double* out,
                               cudaStream_t s);

// Setup construction kernels (kern_setup.cu); asynchronous on s.
cudaError_t build_setup_levels(int n_lev, double p_top, double p_bot, const TablesDev* d_tab, LevelDev* d_levels,
                               cudaStream_t s);
cudaError_t build_quadratures(int n_mu, int n_gll, double* d_out, cudaStream_t s);
cudaError_t build_w_rows(const TablesDev* d_tab, int nu_first, int n_nu, double R, int n_bins, const double* d_edges,
                         int* d_lo, int* d_hi, double* d_invz, int* d_bin, int* d_rowinfo, int* d_err,
                         cudaStream_t s);
cudaError_t build_w_values(const TablesDev* d_tab, int nu_first, double R, int n_bins, const int* d_lo,
                           const int* d_hi, const double* d_invz, const int* d_rowinfo, const long long* d_rowptr,
                           float* d_w32, double* d_w64, cudaStream_t s);
cudaError_t build_nu_pairs(const TablesDev* d_tab, int tile0, int n_tiles, float4* d_nu, float2* d_c1n, cudaStream_t s);
cudaError_t build_level_cache(const TablesDev* d_tab, const SetupDev& h, float* d_lvl, cudaStream_t s);
cudaError_t quantise_fp16(const double* d_src, __half* d_dst, long long rows, int n_nu, int nu_pad, double off,
                          cudaStream_t s);
cudaError_t copy_pad_fp64(const double* d_src, double* d_dst, long long rows, int n_nu, int nu_pad,
                          cudaStream_t s);

}  // namespace hr2
