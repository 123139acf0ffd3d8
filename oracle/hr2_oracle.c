/*
 * hr2_oracle.c -- plain double-precision CPU oracle of the Helios-r2 emission
 * forward model and its Gaussian log-likelihood (Kitzmann et al. 2020,
 * "Helios-r2: A new Bayesian, open-source retrieval model for brown dwarfs
 * and exoplanet atmospheres", Sects. 2 and 3).
 *
 * TEST INFRASTRUCTURE ONLY.  This is the independent reference the CUDA
 * library is checked against.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load it.  It shares no code, header,
 * table or constant with the CUDA library, and the CUDA library never calls
 * it.
 *
 * Style: every function is a direct transcription of the definition it cites,
 * in double precision, in the order the text gives, with no blocking, fusion,
 * precomputed operators or fast-math.  Where the paper is silent or garbled
 * the reading taken is stated at the function (readings R1..R13).
 *
 * Units are cgs throughout (Sect. 4, footnote on log g); pressures enter in
 * bar and are converted to dyn cm^-2; wavenumbers are in cm^-1.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---- physical constants (CODATA 2018 exact/recommended values, cgs) ---- */
#define OR_H      6.62607015e-27      /* Planck constant, erg s            */
#define OR_C      2.99792458e10       /* speed of light, cm s^-1           */
#define OR_KB     1.380649e-16        /* Boltzmann constant, erg K^-1      */
#define OR_AMU    1.66053906660e-24   /* atomic mass unit, g               */
#define OR_PARSEC 3.0856775814913673e18 /* cm                              */
#define OR_BAR    1.0e6               /* dyn cm^-2 per bar                 */
#define OR_M_H2   2.01588             /* u                                 */
#define OR_M_HE   4.002602            /* u                                 */
#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ---- parameter vector layout (one row per sample) ----
 * 0 log10 g (cgs), 1 calibration factor f, 2 distance d in parsec,
 * 3..18 finite-element nodal temperatures, bottom node first (Sect. 2.5.1),
 * 19..34 log10 volume mixing ratios of the setup's absorbers (Sect. 2.4),
 * 35..37 gray cloud layer (Appendix, "Impact of a gray cloud layer"):
 * log10 of its optical depth, log10 of its top pressure in bar, log10 of
 * the fraction f_c (reading R16: the layer spans p_top .. p_top / f_c). */
#define OR_P_LOGG  0
#define OR_P_F     1
#define OR_P_DIST  2
#define OR_P_T0    3
#define OR_P_X0    19
#define OR_P_CLOUD 35
#define OR_NPARAM  38
#define OR_MAX_T   16
#define OR_MAX_SP  16
#define OR_MAX_MU  16

typedef struct {
  /* opacity tables: dequantised log10 cross-sections (cm^2 per molecule) */
  int n_species_tab, n_T, n_p, n_nu_tab;
  const double* T_grid;         /* [n_T] K, strictly ascending                */
  const double* log10p_grid;    /* [n_p] log10(p / bar), strictly ascending   */
  double nu0, dnu;              /* table grid nu_i = nu0 + i*dnu (cm^-1)      */
  const double* log10_sigma;    /* [n_species_tab][n_T][n_p][n_nu_tab]       */
  const double* log10_cia_h2h2; /* [n_T][n_nu_tab] log10 cm^5, or NULL        */
  const double* log10_cia_h2he; /* [n_T][n_nu_tab] log10 cm^5, or NULL        */
  const double* species_mass;   /* [n_species_tab] molecular mass in u        */
  /* spectral / atmospheric setup */
  int nu_first, n_nu;           /* table indices [nu_first, nu_first+n_nu)    */
  int n_layers;                 /* L layers, L+1 levels                       */
  double p_top, p_bot;          /* bar                                        */
  int n_used;                   /* absorbers used by this setup               */
  const int* species;           /* [n_used] indices into the table            */
  int n_mu;                     /* Gauss angle nodes in (0,1]                 */
  int fe_elements, fe_order;    /* K_e, q                                     */
  double resolving_power;       /* R = nu/FWHM; <= 0: no instrument profile   */
  int n_bins;
  const double* bin_edges;      /* [n_bins+1] cm^-1, ascending                */
  double r_he;                  /* n_He / n_H2 of the filling gas             */
  double radius_cm;             /* R_star in the radius-distance relation        */
  int interp;                   /* OR_INTERP_LOG10 or OR_INTERP_LINEAR        */
  int profile;                  /* OR_PROFILE_FE or OR_PROFILE_MILNE          */
  int n_hopf;                   /* Hopf function table (Milne profile only):  */
  const double* hopf_tau;       /*   [n_hopf] ascending optical depths         */
  const double* hopf_q;         /*   [n_hopf] q(tau) at those depths            */
  int cloud;                    /* 1: gray cloud layer from parameters 35..37 */
  int sc_order;                 /* 1 linear (default), 2 parabolic source      */
} or_model;

/* Temperature profile (Sect. 2.5): OR_PROFILE_FE, the finite-element profile
 * of Sect. 2.5.1 (parameters 3.. are the nodal temperatures), or
 * OR_PROFILE_MILNE, Milne's gray radiative-equilibrium profile
 * T^4 = 3/4 Tbar^4 [tau_R + q(tau_R)] with the exact Hopf function q
 * (parameter 3 is Tbar_eff in K, parameter 4 is log10 of the Rosseland
 * opacity kappa_R in cm^2 g^-1; reading R15: tau_R = kappa_R p / g, the
 * hydrostatic optical depth of a constant opacity). */
#define OR_PROFILE_FE    0
#define OR_PROFILE_MILNE 1

/* Interpolation space of the opacity tables (Sect. 2.8 says the tables are
 * interpolated but not in which quantity).  OR_INTERP_LOG10 (reading R3, the
 * default) interpolates log10 sigma and exponentiates the result;
 * OR_INTERP_LINEAR interpolates the cross-sections (and CIA coefficients)
 * themselves, with the same cells and weights. */
#define OR_INTERP_LOG10  0
#define OR_INTERP_LINEAR 1

/* ======================================================================
 * Quadratures
 * ====================================================================== */

/* Legendre polynomial P_n(x) and its derivative by the three-term recurrence. */
static void or_legendre(int n, double x, double* pn, double* dpn) {
  double p0 = 1.0, p1 = x;
  if (n == 0) { *pn = 1.0; *dpn = 0.0; return; }
  for (int k = 2; k <= n; ++k) {
    double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
    p0 = p1; p1 = p2;
  }
  *pn = p1;
  *dpn = n * (x * p1 - p0) / (x * x - 1.0);
}

/* Gauss-Legendre nodes and weights mapped from [-1,1] onto [0,1] (reading R6:
 * the "Gauss quadrature scheme" of Sect. 2.1 is Gauss-Legendre in mu on
 * [0,1]).  Newton iteration on P_n from the Chebyshev-like first guess.
 * Returns 0, or -1 for n outside 1..OR_MAX_MU. */
int or_gauss_legendre01(int n, double* mu, double* w) {
  if (n < 1 || n > OR_MAX_MU) return -1;
  for (int i = 0; i < n; ++i) {
    double x = cos(M_PI * (i + 0.75) / (n + 0.5));
    double pn, dpn;
    for (int it = 0; it < 100; ++it) {
      or_legendre(n, x, &pn, &dpn);
      double dx = pn / dpn;
      x -= dx;
      if (fabs(dx) < 1e-16) break;
    }
    or_legendre(n, x, &pn, &dpn);
    double wx = 2.0 / ((1.0 - x * x) * dpn * dpn);
    /* x descends with i; store ascending mu */
    mu[n - 1 - i] = 0.5 * (x + 1.0);
    w[n - 1 - i] = 0.5 * wx;
  }
  return 0;
}

/* Gauss-Lobatto points on the reference element [0,1] (Sect. 2.5.1): the two
 * end points plus the roots of P'_{np-1}, found by Newton on P'_{N} using the
 * Legendre differential equation for P''.  Returns 0 or -1. */
int or_gauss_lobatto01(int np, double* xi) {
  if (np < 2 || np > OR_MAX_T) return -1;
  int N = np - 1;
  xi[0] = 0.0;
  xi[np - 1] = 1.0;
  for (int i = 1; i < N; ++i) {
    double x = -cos(M_PI * i / N);   /* Chebyshev-Gauss-Lobatto first guess */
    for (int it = 0; it < 100; ++it) {
      double pn, dpn;
      or_legendre(N, x, &pn, &dpn);
      double d2pn = (2.0 * x * dpn - N * (N + 1.0) * pn) / (1.0 - x * x);
      double dx = dpn / d2pn;
      x -= dx;
      if (fabs(dx) < 1e-16) break;
    }
    xi[i] = 0.5 * (x + 1.0);
  }
  return 0;
}

/* Lagrange basis polynomial l_i through the np points xi, Eq. (13). */
double or_lagrange(int np, const double* xi, int i, double x) {
  double v = 1.0;
  for (int j = 0; j < np; ++j)
    if (j != i) v *= (x - xi[j]) / (xi[i] - xi[j]);
  return v;
}

/* ======================================================================
 * Temperature profile, Sect. 2.5.1, Eqs. (12)-(16)
 * ====================================================================== */

/* Continuous finite-element profile.  K_e elements of order q split the
 * modelled range of log p evenly; x in [0,1] is the position from the bottom
 * (x = 0, p = p_bot) to the top (x = 1, p = p_top).  Global dof 0 is the
 * bottom temperature T_1 of Sect. 2.5.1; element k owns dofs k*q .. k*q+q,
 * sharing its end dofs with its neighbours (continuous formulation), so
 * N_T = K_e q + 1 (Eq. 16).  Within an element the local coordinate runs
 * over [0,1] with Gauss-Lobatto nodes (reading R13 for the direction). */
double or_fe_temperature(int Ke, int q, const double* Tnodes, double x) {
  double xi[OR_MAX_T];
  or_gauss_lobatto01(q + 1, xi);
  int k = (int)floor(x * Ke);
  if (k < 0) k = 0;
  if (k > Ke - 1) k = Ke - 1;
  double local = x * Ke - k;
  double T = 0.0;
  for (int i = 0; i <= q; ++i) T += Tnodes[k * q + i] * or_lagrange(q + 1, xi, i, local);
  return T;
}

/* Nodal temperatures from the retrieved bottom temperature T_1 and the
 * ratios b_i (Sect. 2.5.1): every node is b times the node below it
 * (reading R12).  b has n_nodes-1 entries. */
void or_nodes_from_b(int n_nodes, double T1, const double* b, double* Tnodes) {
  Tnodes[0] = T1;
  for (int i = 1; i < n_nodes; ++i) Tnodes[i] = b[i - 1] * Tnodes[i - 1];
}

/* Hopf function q(tau) from the model's table: cubic Lagrange interpolation
 * through the four nearest nodes (the stencil slides inward at the ends),
 * constant beyond the table's ends. */
double or_hopf(const or_model* m, double tau) {
  const double* t = m->hopf_tau;
  const double* q = m->hopf_q;
  int n = m->n_hopf;
  if (tau <= t[0]) return q[0];
  if (tau >= t[n - 1]) return q[n - 1];
  int k = 0;                               /* t[k] < tau <= t[k+1] */
  while (t[k + 1] < tau) ++k;
  int k0 = k - 1;
  if (k0 < 0) k0 = 0;
  if (k0 > n - 4) k0 = n - 4;
  double sum = 0.0;
  for (int a = 0; a < 4; ++a) {
    double l = 1.0;
    for (int b = 0; b < 4; ++b)
      if (b != a) l *= (tau - t[k0 + b]) / (t[k0 + a] - t[k0 + b]);
    sum += l * q[k0 + a];
  }
  return sum;
}

/* Milne's profile (Sect. 2.5): T^4 = 3/4 Tbar^4 [tau_R + q(tau_R)] with
 * tau_R = kappa_R p / g (reading R15), p in dyn cm^-2, g in cm s^-2. */
double or_milne_temperature(const or_model* m, double Tbar, double log10_kappa, double p, double g) {
  double tau = pow(10.0, log10_kappa) * p / g;
  return pow(0.75 * pow(Tbar, 4.0) * (tau + or_hopf(m, tau)), 0.25);
}

/* ======================================================================
 * Source function, Sect. 2.1, Eq. (2)
 * ====================================================================== */

/* Planck function per unit wavenumber, erg s^-1 cm^-2 sr^-1 (cm^-1)^-1. */
double or_planck(double nu, double T) {
  double x = OR_H * OR_C * nu / (OR_KB * T);
  return 2.0 * OR_H * OR_C * OR_C * nu * nu * nu / expm1(x);
}

/* ======================================================================
 * Short characteristics, Sect. 2.1, Eqs. (4)-(8)
 * ====================================================================== */

/* Emergent intensity at the top of the atmosphere along mu.
 * Levels j = 0 (top) .. L (bottom); layer l lies between levels l and l+1 and
 * has optical depth dtau[l]; S[j] is the source function at level j; the ray
 * enters the bottom level with intensity I_bottom (reading R5: B(T_L)).
 * Each layer: I_l = I_{l+1} e^{-D} + beta S_l + gamma S_{l+1}, D = dtau/mu,
 * with beta = 1 - (1-e^{-D})/D for the near (upper) level and
 * gamma = (1-e^{-D})/D - e^{-D} for the far (deeper) level: the exact
 * integral of a linearly varying source (reading R1; the printed gamma of
 * Eq. 6 has the sign of its e^{-D} terms swapped, which would make a
 * transparent isothermal layer emit twice its Planck intensity). */
double or_sc_intensity(int L, const double* dtau, const double* S, double I_bottom, double mu) {
  double I = I_bottom;
  for (int l = L - 1; l >= 0; --l) {
    double D = dtau[l] / mu;
    double e = exp(-D);
    double q = (D > 0.0) ? -expm1(-D) / D : 1.0;
    double beta = 1.0 - q;
    double gamma = q - e;
    I = I * e + beta * S[l] + gamma * S[l + 1];
  }
  return I;
}

/* M_k(D) = int_0^D t^k e^{-t} dt, k = 0, 1, 2: by the power series
 * sum_n (-1)^n D^{k+n+1} / (n! (k+n+1)) for D < 1/2 (no cancellation for thin
 * layers), else by the closed forms M_0 = 1 - e^{-D}, M_1 = M_0 - D e^{-D},
 * M_2 = 2 M_1 - D^2 e^{-D}. */
static void or_moments(double D, double* M0, double* M1, double* M2) {
  if (D < 0.5) {
    double s[3] = {0.0, 0.0, 0.0};
    double term = D;                            /* (-1)^n D^{n+1} / n! */
    for (int n = 0; n < 60; ++n) {
      for (int k = 0; k < 3; ++k) s[k] += term * pow(D, k) / (double)(k + n + 1);
      term *= -D / (double)(n + 1);
      if (fabs(term) < 1e-30) break;
    }
    *M0 = s[0]; *M1 = s[1]; *M2 = s[2];
  } else {
    double e = exp(-D);
    *M0 = -expm1(-D);
    *M1 = *M0 - D * e;
    *M2 = 2.0 * *M1 - D * D * e;
  }
}

/* Parabolic short characteristics (Sect. 2.1: higher-order interpolants of
 * the source, after Olson & Kunasz 1987), written here from the definition:
 * along the ray, t is the optical depth below point l; over layer l (t from 0
 * to D_u) the source is the parabola through S_{l-1} (t = -D_d), S_l (t = 0)
 * and S_{l+1} (t = D_u), and I_l = I_{l+1} e^{-D_u} + int_0^{D_u} S(t) e^{-t} dt.
 * In Taylor form at t = 0, S(t) = S_l + c1 t + c2 t^2 with the divided
 * differences d_u = (S_{l+1} - S_l)/D_u, d_d = (S_l - S_{l-1})/D_d,
 * c2 = (d_u - d_d)/(D_u + D_d), c1 = d_u - c2 D_u, so that
 *   int_0^{D_u} S e^{-t} dt = S_l M_0 + c1 M_1 + c2 M_2.
 * (The same integral as the Lagrange-weight form, without its cancellation
 * when D_d << D_u.)  The top layer (no point above) and a layer under a
 * zero-thickness layer use the linear source (c2 = 0, c1 = d_u). */
double or_sc_intensity_parabolic(int L, const double* dtau, const double* S, double I_bottom, double mu) {
  double I = I_bottom;
  for (int l = L - 1; l >= 0; --l) {
    double Du = dtau[l] / mu;
    if (!(Du > 0.0)) continue;                  /* a transparent layer changes nothing */
    double Dd = (l > 0) ? dtau[l - 1] / mu : 0.0;
    double M0, M1, M2;
    or_moments(Du, &M0, &M1, &M2);
    double du = (S[l + 1] - S[l]) / Du;
    double c2 = 0.0, c1 = du;
    if (Dd > 0.0) {
      double dd = (S[l] - S[l - 1]) / Dd;
      c2 = (du - dd) / (Du + Dd);
      c1 = du - c2 * Du;
    }
    I = I * exp(-Du) + S[l] * M0 + c1 * M1 + c2 * M2;
  }
  return I;
}

/* Outgoing flux F+ = 2 pi int_0^1 I mu dmu by Gauss-Legendre, Eq. (8). */
double or_sc_flux(int L, const double* dtau, const double* S, double I_bottom, int n_mu) {
  double mu[OR_MAX_MU], w[OR_MAX_MU];
  or_gauss_legendre01(n_mu, mu, w);
  double F = 0.0;
  for (int k = 0; k < n_mu; ++k) F += w[k] * mu[k] * or_sc_intensity(L, dtau, S, I_bottom, mu[k]);
  return 2.0 * M_PI * F;
}

/* The same with the parabolic scheme. */
double or_sc_flux_parabolic(int L, const double* dtau, const double* S, double I_bottom, int n_mu) {
  double mu[OR_MAX_MU], w[OR_MAX_MU];
  or_gauss_legendre01(n_mu, mu, w);
  double F = 0.0;
  for (int k = 0; k < n_mu; ++k) F += w[k] * mu[k] * or_sc_intensity_parabolic(L, dtau, S, I_bottom, mu[k]);
  return 2.0 * M_PI * F;
}

/* ======================================================================
 * Opacity interpolation (Sect. 2.8) -- reading R3: bilinear in (T, log10 p)
 * on log10 sigma, clamped to the table edges.
 * ====================================================================== */

/* Cell index i (grid[i] <= v <= grid[i+1]) and weight of grid[i+1]; values
 * outside the grid are clamped to its end points. */
static void or_cell(const double* grid, int n, double v, int* i, double* w) {
  if (v <= grid[0]) { *i = 0; *w = 0.0; return; }
  if (v >= grid[n - 1]) { *i = n - 2; *w = 1.0; return; }
  int k = 0;
  while (grid[k + 1] < v) ++k;
  *i = k;
  *w = (v - grid[k]) / (grid[k + 1] - grid[k]);
}

/* log10 sigma of table species s at (T, log10 p) and table index inu. */
double or_log10_sigma(const or_model* m, int s, double T, double log10p, int inu) {
  int a, b;
  double wT, wp;
  or_cell(m->T_grid, m->n_T, T, &a, &wT);
  or_cell(m->log10p_grid, m->n_p, log10p, &b, &wp);
  const double* tab = m->log10_sigma + (size_t)s * m->n_T * m->n_p * m->n_nu_tab;
#define OR_TAB(ia, ib) tab[((size_t)(ia) * m->n_p + (ib)) * m->n_nu_tab + inu]
  double v = (1.0 - wT) * (1.0 - wp) * OR_TAB(a, b) + wT * (1.0 - wp) * OR_TAB(a + 1, b) +
             (1.0 - wT) * wp * OR_TAB(a, b + 1) + wT * wp * OR_TAB(a + 1, b + 1);
#undef OR_TAB
  return v;
}

/* log10 of a collision-induced absorption coefficient (cm^5), linear in T. */
double or_log10_cia(const or_model* m, const double* cia, double T, int inu) {
  int a;
  double wT;
  or_cell(m->T_grid, m->n_T, T, &a, &wT);
  return (1.0 - wT) * cia[(size_t)a * m->n_nu_tab + inu] + wT * cia[(size_t)(a + 1) * m->n_nu_tab + inu];
}

/* Cross-section (cm^2) of table species s at (T, log10 p), table index inu,
 * in the setup's interpolation space: 10^(bilinear log10 sigma), or the
 * bilinear combination of the four corner cross-sections 10^(log10 sigma). */
double or_sigma(const or_model* m, int s, double T, double log10p, int inu) {
  if (m->interp != OR_INTERP_LINEAR) return pow(10.0, or_log10_sigma(m, s, T, log10p, inu));
  int a, b;
  double wT, wp;
  or_cell(m->T_grid, m->n_T, T, &a, &wT);
  or_cell(m->log10p_grid, m->n_p, log10p, &b, &wp);
  const double* tab = m->log10_sigma + (size_t)s * m->n_T * m->n_p * m->n_nu_tab;
#define OR_SIG(ia, ib) pow(10.0, tab[((size_t)(ia) * m->n_p + (ib)) * m->n_nu_tab + inu])
  double v = (1.0 - wT) * (1.0 - wp) * OR_SIG(a, b) + wT * (1.0 - wp) * OR_SIG(a + 1, b) +
             (1.0 - wT) * wp * OR_SIG(a, b + 1) + wT * wp * OR_SIG(a + 1, b + 1);
#undef OR_SIG
  return v;
}

/* Collision-induced absorption coefficient (cm^5) at T, table index inu, in
 * the setup's interpolation space (linear in T either way). */
double or_cia_coeff(const or_model* m, const double* cia, double T, int inu) {
  if (m->interp != OR_INTERP_LINEAR) return pow(10.0, or_log10_cia(m, cia, T, inu));
  int a;
  double wT;
  or_cell(m->T_grid, m->n_T, T, &a, &wT);
  return (1.0 - wT) * pow(10.0, cia[(size_t)a * m->n_nu_tab + inu]) +
         wT * pow(10.0, cia[(size_t)(a + 1) * m->n_nu_tab + inu]);
}

/* ======================================================================
 * Per-sample state
 * ====================================================================== */

typedef struct {
  int valid;
  int L;
  double p[1024];          /* level pressure, dyn cm^-2 (j = 0 top)         */
  double log10p_bar[1024];
  double T[1024];          /* level temperature, K                          */
  double x[OR_MAX_SP];     /* absorber volume mixing ratios                 */
  double x_h2, x_he;
  double mmw;              /* mean molecular weight, u                      */
  double g;                /* surface gravity, cm s^-2                      */
  double scale;            /* f (R_star / d)^2, Eq. (9)                        */
  double tau_cloud[1024];  /* gray cloud optical depth of each layer          */
} or_state;

#define OR_MAX_LEVELS 1024

/* Level grid equidistant in log p (Sect. 2), T profile (Sect. 2.5.1), free
 * chemistry with H2/He filling the remainder at the ratio r_he (Sect. 2.4,
 * reading R4), g and the radius-distance factor.  Returns 1 if the sample is
 * physically valid, 0 otherwise (non-positive or non-finite T, f, d, or
 * absorber mixing ratios summing to 1 or more). */
int or_prepare(const or_model* m, const double* theta, or_state* st) {
  int L = m->n_layers;
  st->L = L;
  st->valid = 0;
  if (L < 1 || L + 1 > OR_MAX_LEVELS) return 0;
  double lt = log10(m->p_top), lb = log10(m->p_bot);
  int Ke = m->fe_elements, q = m->fe_order;
  int ok = 1;
  double grav = pow(10.0, theta[OR_P_LOGG]);
  for (int j = 0; j <= L; ++j) {
    double lp = lt + (lb - lt) * (double)j / (double)L;
    st->log10p_bar[j] = lp;
    st->p[j] = pow(10.0, lp) * OR_BAR;
    double T;
    if (m->profile == OR_PROFILE_MILNE)
      T = or_milne_temperature(m, theta[OR_P_T0], theta[OR_P_T0 + 1], st->p[j], grav);
    else
      T = or_fe_temperature(Ke, q, theta + OR_P_T0, (double)(L - j) / (double)L);
    st->T[j] = T;
    if (!(T > 0.0) || !isfinite(T)) ok = 0;
  }
  double sumx = 0.0;
  for (int s = 0; s < m->n_used; ++s) {
    double lx = theta[OR_P_X0 + s];
    if (!isfinite(lx)) ok = 0;
    st->x[s] = pow(10.0, lx);
    sumx += st->x[s];
  }
  if (!(sumx < 1.0)) ok = 0;
  st->x_h2 = (1.0 - sumx) / (1.0 + m->r_he);
  st->x_he = m->r_he * st->x_h2;
  double mmw = st->x_h2 * OR_M_H2 + st->x_he * OR_M_HE;
  for (int s = 0; s < m->n_used; ++s) mmw += st->x[s] * m->species_mass[m->species[s]];
  st->mmw = mmw;
  st->g = pow(10.0, theta[OR_P_LOGG]);
  double f = theta[OR_P_F], d = theta[OR_P_DIST] * OR_PARSEC;
  if (!(f > 0.0) || !(d > 0.0) || !isfinite(f) || !isfinite(d) || !isfinite(st->g)) ok = 0;
  st->scale = f * (m->radius_cm / d) * (m->radius_cm / d);
  /* Gray cloud (reading R17): optical depth tau_c spread evenly in pressure
   * over [p_top, p_top / f_c] (a constant gray extinction per unit mass in
   * hydrostatic equilibrium); a layer gets tau_c times the fraction of that
   * pressure range it covers. */
  for (int l = 0; l < L; ++l) st->tau_cloud[l] = 0.0;
  if (m->cloud) {
    double tc = pow(10.0, theta[OR_P_CLOUD]);
    double pt = pow(10.0, theta[OR_P_CLOUD + 1]) * OR_BAR;
    double fc = pow(10.0, theta[OR_P_CLOUD + 2]);
    if (!isfinite(tc) || !(tc >= 0.0) || !(pt > 0.0) || !isfinite(pt) || !(fc > 0.0) || !(fc <= 1.0)) ok = 0;
    double pb = pt / fc;
    if (ok && pb > pt) {
      for (int l = 0; l < L; ++l) {
        double lo = fmax(st->p[l], pt), hi = fmin(st->p[l + 1], pb);
        if (hi > lo) st->tau_cloud[l] = tc * (hi - lo) / (pb - pt);
      }
    }
  }
  st->valid = ok;
  return ok;
}

/* Absorption coefficient per molecule (cm^2) at level j and table index inu:
 * the abundance-weighted sum of the absorbers' cross-sections plus the H2-H2
 * and H2-He collision-induced terms x_H2 x_X n k(T, nu) (Sects. 2.3, 2.8). */
double or_chi(const or_model* m, const or_state* st, int j, int inu) {
  double chi = 0.0;
  for (int s = 0; s < m->n_used; ++s)
    chi += st->x[s] * or_sigma(m, m->species[s], st->T[j], st->log10p_bar[j], inu);
  double n_tot = st->p[j] / (OR_KB * st->T[j]);
  if (m->log10_cia_h2h2)
    chi += st->x_h2 * st->x_h2 * n_tot * or_cia_coeff(m, m->log10_cia_h2h2, st->T[j], inu);
  if (m->log10_cia_h2he)
    chi += st->x_h2 * st->x_he * n_tot * or_cia_coeff(m, m->log10_cia_h2he, st->T[j], inu);
  return chi;
}

/* Top-of-atmosphere outgoing flux F+ (Eq. 8, not yet scaled by Eq. 9) at the
 * setup's wavenumber index k (table index nu_first + k).
 * Layer optical depth (reading R2): trapezoid of the level coefficients in
 * pressure with hydrostatic column mass dm = dp / g, i.e.
 * dtau_l = (chi_l + chi_{l+1}) / 2 * (p_{l+1} - p_l) / (mmw m_u g). */
double or_top_flux(const or_model* m, const or_state* st, int k) {
  int L = st->L;
  int inu = m->nu_first + k;
  double nu = m->nu0 + (double)inu * m->dnu;
  double chi[OR_MAX_LEVELS], S[OR_MAX_LEVELS], dtau[OR_MAX_LEVELS];
  for (int j = 0; j <= L; ++j) {
    chi[j] = or_chi(m, st, j, inu);
    S[j] = or_planck(nu, st->T[j]);
  }
  double colfac = 1.0 / (st->mmw * OR_AMU * st->g);
  for (int l = 0; l < L; ++l)
    dtau[l] = 0.5 * (chi[l] + chi[l + 1]) * (st->p[l + 1] - st->p[l]) * colfac + st->tau_cloud[l];
  if (m->sc_order == 2) return or_sc_flux_parabolic(L, dtau, S, S[L], m->n_mu);
  return or_sc_flux(L, dtau, S, S[L], m->n_mu);
}

/* Wavenumber of setup point k. */
static double or_nu(const or_model* m, int k) { return m->nu0 + (double)(m->nu_first + k) * m->dnu; }

/* Instrument profile, Sect. 2.7, Eq. (17) (reading R8): Gaussian of standard
 * deviation sigma = nu / (R 2 sqrt(2 ln 2)) centred on the output point,
 * truncated at |x - nu| = 5 sigma and renormalised over the points kept.
 * Fin/Fout are over the setup's n_nu points. */
void or_convolve(const or_model* m, const double* Fin, double* Fout) {
  int n = m->n_nu;
  if (!(m->resolving_power > 0.0)) {
    for (int i = 0; i < n; ++i) Fout[i] = Fin[i];
    return;
  }
  for (int i = 0; i < n; ++i) {
    double nui = or_nu(m, i);
    double sig = nui / (m->resolving_power * 2.0 * sqrt(2.0 * log(2.0)));
    double num = 0.0, den = 0.0;
    for (int j = 0; j < n; ++j) {
      double dx = or_nu(m, j) - nui;
      if (fabs(dx) <= 5.0 * sig) {
        double g = exp(-dx * dx / (2.0 * sig * sig));
        num += g * Fin[j];
        den += g;
      }
    }
    Fout[i] = num / den;
  }
}

/* Binning to the observed bins (Sect. 2.8, reading R9): the mean of the
 * points with edge_b <= nu < edge_{b+1}, the last bin closed.  Returns the
 * number of empty bins (their value is NaN). */
int or_bin(const or_model* m, const double* F, double* bins) {
  int empty = 0;
  for (int b = 0; b < m->n_bins; ++b) {
    double lo = m->bin_edges[b], hi = m->bin_edges[b + 1];
    double sum = 0.0;
    int cnt = 0;
    for (int i = 0; i < m->n_nu; ++i) {
      double nu = or_nu(m, i);
      int in = (nu >= lo) && ((b == m->n_bins - 1) ? (nu <= hi) : (nu < hi));
      if (in) { sum += F[i]; ++cnt; }
    }
    if (cnt == 0) { bins[b] = NAN; ++empty; }
    else bins[b] = sum / cnt;
  }
  return empty;
}

/* Full forward model of one sample: F+ at every setup point (optional
 * output, unscaled), then F = F+ f (R_star/d)^2 (Eq. 9), the instrument profile
 * and the binning.  Invalid samples give NaN bins; returns validity. */
int or_forward(const or_model* m, const double* theta, double* bins, double* Ftop_or_null) {
  or_state* st = (or_state*)malloc(sizeof(or_state));
  int ok = or_prepare(m, theta, st);
  int n = m->n_nu;
  double* F = (double*)malloc(sizeof(double) * n);
  double* Fc = (double*)malloc(sizeof(double) * n);
  for (int k = 0; k < n; ++k) {
    double Ft = ok ? or_top_flux(m, st, k) : NAN;
    if (Ftop_or_null) Ftop_or_null[k] = Ft;
    F[k] = Ft * st->scale;
  }
  if (ok) {
    or_convolve(m, F, Fc);
    or_bin(m, Fc, bins);
  } else {
    for (int b = 0; b < m->n_bins; ++b) bins[b] = NAN;
  }
  free(Fc); free(F); free(st);
  return ok;
}

/* Effective temperature (Sect. 2.6): the outgoing flux F+ at the top of the
 * atmosphere (before the distance dilution of Eq. 9), integrated over the
 * setup's wavenumbers by the trapezoid rule, converted with the
 * Stefan-Boltzmann law F = sigma T_eff^4, sigma = 2 pi^5 k^4 / (15 h^3 c^2). */
double or_effective_temperature(const or_model* m, const double* Ftop) {
  double F = 0.0;
  for (int k = 0; k + 1 < m->n_nu; ++k) F += 0.5 * (Ftop[k] + Ftop[k + 1]) * m->dnu;
  double sigma = 2.0 * pow(M_PI, 5) * pow(OR_KB, 4) / (15.0 * pow(OR_H, 3) * OR_C * OR_C);
  return pow(F / sigma, 0.25);
}

/* F+ (unscaled) at a chosen list of setup indices: the same per-point
 * computation as or_forward, for sampled comparisons on large setups. */
int or_top_flux_at(const or_model* m, const double* theta, int n_idx, const int* idx, double* Ftop) {
  or_state* st = (or_state*)malloc(sizeof(or_state));
  int ok = or_prepare(m, theta, st);
  for (int i = 0; i < n_idx; ++i) Ftop[i] = ok ? or_top_flux(m, st, idx[i]) : NAN;
  free(st);
  return ok;
}

/* Chosen bins only: evaluates F+ on every setup point that can reach one of
 * the selected bins through the 5-sigma instrument profile, then applies the
 * same convolution and binning definitions.  For sampled comparisons. */
int or_bins_at(const or_model* m, const double* theta, int n_sel, const int* sel, double* out) {
  or_state* st = (or_state*)malloc(sizeof(or_state));
  int ok = or_prepare(m, theta, st);
  int n = m->n_nu;
  double* F = (double*)malloc(sizeof(double) * n);
  char* need = (char*)calloc(n, 1);
  double c = (m->resolving_power > 0.0) ? 5.0 / (m->resolving_power * 2.0 * sqrt(2.0 * log(2.0))) : 0.0;
  for (int t = 0; t < n_sel; ++t) {
    double lo = m->bin_edges[sel[t]], hi = m->bin_edges[sel[t] + 1];
    /* a point i in [lo,hi] sees j with |nu_j - nu_i| <= 5 sigma_i <= c*hi */
    for (int j = 0; j < n; ++j) {
      double nu = or_nu(m, j);
      if (nu >= lo - c * hi - m->dnu && nu <= hi + c * hi + m->dnu) need[j] = 1;
    }
  }
  for (int j = 0; j < n; ++j) F[j] = (ok && need[j]) ? or_top_flux(m, st, j) * st->scale : 0.0;
  for (int t = 0; t < n_sel; ++t) {
    int b = sel[t];
    double lo = m->bin_edges[b], hi = m->bin_edges[b + 1];
    double sum = 0.0;
    int cnt = 0;
    for (int i = 0; i < n; ++i) {
      double nui = or_nu(m, i);
      int in = (nui >= lo) && ((b == m->n_bins - 1) ? (nui <= hi) : (nui < hi));
      if (!in) continue;
      double v;
      if (m->resolving_power > 0.0) {
        double sig = nui / (m->resolving_power * 2.0 * sqrt(2.0 * log(2.0)));
        double num = 0.0, den = 0.0;
        for (int j = 0; j < n; ++j) {
          double dx = or_nu(m, j) - nui;
          if (fabs(dx) <= 5.0 * sig) {
            double g = exp(-dx * dx / (2.0 * sig * sig));
            num += g * F[j];
            den += g;
          }
        }
        v = num / den;
      } else {
        v = F[i];
      }
      sum += v;
      ++cnt;
    }
    out[t] = (ok && cnt > 0) ? sum / cnt : NAN;
  }
  free(need); free(F); free(st);
  return ok;
}

/* ======================================================================
 * Likelihood, Sect. 3.1 Eq. (19) and Sect. 3.3 Eqs. (22)-(23)
 * ====================================================================== */

/* ln L = sum_j [ -(D_j - D_m,j)^2 / (2 s_j^2) - ln(2 pi s_j^2) / 2 ] with
 * s_j^2 = sigma_j^2 (+ 10^eps when error inflation is used, i.e. when
 * log_eps is finite).  Any non-finite model bin gives -inf. */
double or_lnL(int n_bins, const double* D, const double* sigma, const double* Dm, double log_eps) {
  double lnL = 0.0;
  for (int j = 0; j < n_bins; ++j) {
    if (!isfinite(Dm[j])) return -INFINITY;
    double s2 = sigma[j] * sigma[j];
    if (isfinite(log_eps)) s2 += pow(10.0, log_eps);
    double r = D[j] - Dm[j];
    lnL += -r * r / (2.0 * s2) - 0.5 * log(2.0 * M_PI * s2);
  }
  return lnL;
}

/* ======================================================================
 * Batch driver (one sample per OpenMP iteration)
 * ====================================================================== */

/* bins: [n][n_bins]; Ftop_or_null: [n][n_nu] or NULL; valid: [n] or NULL.
 * n_threads <= 0 uses the OpenMP default.  Returns the thread count used. */
int or_forward_batch(const or_model* m, int n, const double* theta, double* bins, double* Ftop_or_null,
                     int* valid_or_null, int n_threads) {
  int used = 1;
#ifdef _OPENMP
  if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel
  {
#pragma omp single
    used = omp_get_num_threads();
  }
#pragma omp parallel for schedule(dynamic, 1)
#endif
  for (int i = 0; i < n; ++i) {
    int ok = or_forward(m, theta + (size_t)i * OR_NPARAM, bins + (size_t)i * m->n_bins,
                        Ftop_or_null ? Ftop_or_null + (size_t)i * m->n_nu : NULL);
    if (valid_or_null) valid_or_null[i] = ok;
  }
  return used;
}

/* Level temperatures of one sample (for the profile pins). */
int or_level_temperatures(const or_model* m, const double* theta, double* T) {
  or_state* st = (or_state*)malloc(sizeof(or_state));
  int ok = or_prepare(m, theta, st);
  for (int j = 0; j <= m->n_layers; ++j) T[j] = st->T[j];
  free(st);
  return ok;
}

/* Layer optical depths of one sample at setup index k (for the scaling pins). */
int or_layer_dtau(const or_model* m, const double* theta, int k, double* dtau) {
  or_state* st = (or_state*)malloc(sizeof(or_state));
  int ok = or_prepare(m, theta, st);
  int L = st->L, inu = m->nu_first + k;
  double colfac = 1.0 / (st->mmw * OR_AMU * st->g);
  double prev = or_chi(m, st, 0, inu);
  for (int l = 0; l < L; ++l) {
    double next = or_chi(m, st, l + 1, inu);
    dtau[l] = 0.5 * (prev + next) * (st->p[l + 1] - st->p[l]) * colfac + st->tau_cloud[l];
    prev = next;
  }
  free(st);
  return ok;
}
