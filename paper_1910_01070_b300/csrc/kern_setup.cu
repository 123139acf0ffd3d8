// kern_setup.cu -- device kernels run once per table or setup creation:
// table quantisation, level grid, quadrature nodes and the combined
// instrument-profile + binning operator W.  All in FP64.
#include <algorithm>

#include "hr2_internal.cuh"

namespace hr2 {

// ---------------------------------------------------------------- tables
__global__ void k_quantise_fp16(const double* __restrict__ src, __half* __restrict__ dst, long long rows, int n_nu,
                                int nu_pad, double off) {
  long long total = rows * (long long)nu_pad;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    long long r = t / nu_pad;
    int c = (int)(t - r * nu_pad);
    // binary16 of (value - offset), round to nearest even
    dst[t] = (c < n_nu) ? __double2half(src[r * n_nu + c] - off) : __double2half(0.0);
  }
}

__global__ void k_copy_pad_fp64(const double* __restrict__ src, double* __restrict__ dst, long long rows, int n_nu,
                                int nu_pad) {
  long long total = rows * (long long)nu_pad;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    long long r = t / nu_pad;
    int c = (int)(t - r * nu_pad);
    dst[t] = (c < n_nu) ? src[r * n_nu + c] : 0.0;
  }
}

cudaError_t quantise_fp16(const double* d_src, __half* d_dst, long long rows, int n_nu, int nu_pad, double off,
                          cudaStream_t s) {
  long long total = rows * (long long)nu_pad;
  int grid = (int)((total + 255) / 256 < 4096 ? (total + 255) / 256 : 4096);
  k_quantise_fp16<<<grid, 256, 0, s>>>(d_src, d_dst, rows, n_nu, nu_pad, off);
  return cudaGetLastError();
}

cudaError_t copy_pad_fp64(const double* d_src, double* d_dst, long long rows, int n_nu, int nu_pad,
                          cudaStream_t s) {
  long long total = rows * (long long)nu_pad;
  int grid = (int)((total + 255) / 256 < 4096 ? (total + 255) / 256 : 4096);
  k_copy_pad_fp64<<<grid, 256, 0, s>>>(d_src, d_dst, rows, n_nu, nu_pad);
  return cudaGetLastError();
}

// ------------------------------------------------------------ quadratures
// Legendre P_n and P'_n at x by the three-term recurrence.
__device__ void legendre_pd(int n, double x, double& p, double& dp) {
  double p0 = 1.0, p1 = x;
  if (n == 0) {
    p = 1.0;
    dp = 0.0;
    return;
  }
  for (int k = 2; k <= n; ++k) {
    double p2 = ((2 * k - 1) * x * p1 - (k - 1) * p0) / k;
    p0 = p1;
    p1 = p2;
  }
  p = p1;
  dp = n * (x * p1 - p0) / (x * x - 1.0);
}

// out = [mu (n_mu, ascending) | w (n_mu) | gll (n_gll)], all on [0,1].
// Gauss-Legendre nodes (angle quadrature of Eq. 8) by Newton on P_n;
// Gauss-Lobatto points of the reference element (Sect. 2.5.1) as the end
// points plus the roots of P'_{n_gll-1}.
__global__ void k_quadratures(int n_mu, int n_gll, double* out) {
  int t = threadIdx.x;
  if (t < n_mu) {
    int n = n_mu;
    int i = t;
    double x = cos(kPi * (i + 0.75) / (n + 0.5));
    double p, dp;
    for (int it = 0; it < 60; ++it) {
      legendre_pd(n, x, p, dp);
      double dx = p / dp;
      x -= dx;
      if (fabs(dx) < 1e-16) break;
    }
    legendre_pd(n, x, p, dp);
    out[n - 1 - i] = 0.5 * (x + 1.0);
    out[n_mu + n - 1 - i] = 1.0 / ((1.0 - x * x) * dp * dp);  // = w_x / 2
  }
  if (t < n_gll) {
    int N = n_gll - 1;
    double v;
    if (t == 0) {
      v = 0.0;
    } else if (t == N) {
      v = 1.0;
    } else {
      double x = -cos(kPi * t / N);
      for (int it = 0; it < 60; ++it) {
        double p, dp;
        legendre_pd(N, x, p, dp);
        double d2p = (2.0 * x * dp - N * (N + 1.0) * p) / (1.0 - x * x);
        double dx = dp / d2p;
        x -= dx;
        if (fabs(dx) < 1e-16) break;
      }
      v = 0.5 * (x + 1.0);
    }
    out[2 * n_mu + t] = v;
  }
}

cudaError_t build_quadratures(int n_mu, int n_gll, double* d_out, cudaStream_t s) {
  k_quadratures<<<1, 32, 0, s>>>(n_mu, n_gll, d_out);
  return cudaGetLastError();
}

// ------------------------------------------------------- Hopf function
// q(tau) of Milne's problem (Sect. 2.5) from Chandrasekhar's closed form
//   q(tau) = 1/sqrt(3) + (1/(2 sqrt 3)) int_0^1 g(mu) (1 - e^{-tau/mu}) dmu,
//   g(mu) = 1 / (H(mu) [(1 - (mu/2) ln((1+mu)/(1-mu)))^2 + (pi mu / 2)^2]),
//   ln H(mu) = -(mu/pi) int_0^{pi/2} ln(1 - th cot th) / (cos^2 th + mu^2 sin^2 th) dth,
// H the H-function of conservative isotropic scattering.  Quadratures
// (Gauss-Legendre): theta = (pi/2) s^2 (128 nodes; removes the log
// singularity at theta = 0); mu in [1/2, 1) as mu = 1 - (1-s)^3 / 2 (32
// nodes; clusters at the log singularity of g at mu = 1) and mu in (0, 1/2]
// as mu = e^{-v} / 2, v in [0, 30] (64 nodes; resolves e^{-tau/mu} down to
// tau ~ 1e-9).  One CTA, FP64, once per setup.
constexpr int kHopfTheta = 128, kHopfMuA = 32, kHopfMuB = 64;

// node i of the n-point Gauss-Legendre rule on [-1, 1] and its weight
__device__ void gauss_legendre_node(int n, int i, double& x, double& w) {
  double p, dp;
  x = cos(kPi * (i + 0.75) / (n + 0.5));
  for (int it = 0; it < 60; ++it) {
    legendre_pd(n, x, p, dp);
    const double dx = p / dp;
    x -= dx;
    if (fabs(dx) < 1e-16) break;
  }
  legendre_pd(n, x, p, dp);
  w = 2.0 / ((1.0 - x * x) * dp * dp);
}

// ln(1 - th cot th), by its series th^2/3 (1 + th^2/15 + 2 th^4/315) for small th
__device__ double ln_one_minus_th_cot(double th) {
  const double t2 = th * th;
  if (th < 0.05) return log(t2 / 3.0) + log1p(t2 / 15.0 + 2.0 * t2 * t2 / 315.0);
  return log(1.0 - th / tan(th));
}

__global__ void __launch_bounds__(256) k_hopf_table(double* q_out) {
  __shared__ double s_th[kHopfTheta], s_wth[kHopfTheta];
  __shared__ double s_mu[kHopfMuA + kHopfMuB], s_wg[kHopfMuA + kHopfMuB];
  __shared__ double s_tail0;
  const int t = threadIdx.x;
  if (t < kHopfTheta) {
    double x, w;
    gauss_legendre_node(kHopfTheta, t, x, w);
    const double sn = 0.5 * (x + 1.0);
    s_th[t] = 0.5 * kPi * sn * sn;
    s_wth[t] = 0.5 * w * kPi * sn;               // ds/2 times dtheta/ds
  }
  __syncthreads();
  if (t < kHopfMuA + kHopfMuB) {
    double x, w, mu, wmu;
    if (t < kHopfMuA) {
      gauss_legendre_node(kHopfMuA, t, x, w);
      const double sn = 0.5 * (x + 1.0), om = 1.0 - sn;
      mu = 1.0 - 0.5 * om * om * om;
      wmu = 0.5 * w * 1.5 * om * om;
    } else {
      gauss_legendre_node(kHopfMuB, t - kHopfMuA, x, w);
      const double v = 15.0 * (x + 1.0);
      mu = 0.5 * exp(-v);
      wmu = 15.0 * w * mu;
    }
    double acc = 0.0;
    for (int k = 0; k < kHopfTheta; ++k) {
      const double th = s_th[k], c = cos(th), sn = sin(th);
      acc += s_wth[k] * ln_one_minus_th_cot(th) / (c * c + mu * mu * sn * sn);
    }
    const double H = exp(-mu / kPi * acc);
    const double a = 1.0 - 0.5 * mu * log((1.0 + mu) / (1.0 - mu));
    s_mu[t] = mu;
    s_wg[t] = wmu / (H * (a * a + 0.25 * kPi * kPi * mu * mu));
  }
  __syncthreads();
  if (t == 0) {
    double z = 0.0;
    for (int k = 0; k < kHopfMuA + kHopfMuB; ++k) z += s_wg[k];
    s_tail0 = z;
  }
  __syncthreads();
  const double lt0 = log(kHopfTau0), du = (log(kHopfTau1) - lt0) / (kHopfN - 1);
  const double c0 = 1.0 / sqrt(3.0), c1 = 0.5 / sqrt(3.0);
  for (int i = t; i < kHopfN; i += blockDim.x) {
    const double tau = exp(lt0 + du * i);
    double tail = 0.0;
    for (int k = 0; k < kHopfMuA + kHopfMuB; ++k) tail += s_wg[k] * exp(-tau / s_mu[k]);
    q_out[i] = c0 + c1 * (s_tail0 - tail);
  }
}

cudaError_t build_hopf_table(double* d_q, cudaStream_t s) {
  k_hopf_table<<<1, 256, 0, s>>>(d_q);
  return cudaGetLastError();
}

// --------------------------------------------------------------- levels
// Level j (0 = top) at log10 p_j = lt + (lb - lt) j / L (equidistant in
// log p, Sect. 2); the p-grid cell of the table that brackets it (clamped to
// the grid ends) and the half pressure thickness of layer j.
__device__ double level_log10p(int j, int L, double lt, double lb) { return lt + (lb - lt) * (double)j / (double)L; }

__global__ void k_levels(int n_lev, double lt, double lb, const TablesDev* tab, LevelDev* lev) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n_lev) return;
  int L = n_lev - 1;
  double lp = level_log10p(j, L, lt, lb);
  double p = pow(10.0, lp) * kBar;
  const double* g = tab->log10p_grid64;
  int np = tab->n_p;
  int b;
  double w;
  if (lp <= g[0]) {
    b = 0;
    w = 0.0;
  } else if (lp >= g[np - 1]) {
    b = np - 2;
    w = 1.0;
  } else {
    b = 0;
    while (g[b + 1] < lp) ++b;
    w = (lp - g[b]) / (g[b + 1] - g[b]);
  }
  double half_dp = 0.0;
  if (j < L) {
    double pn = pow(10.0, level_log10p(j + 1, L, lt, lb)) * kBar;
    half_dp = 0.5 * (pn - p);
  }
  LevelDev d;
  d.pcell = b;
  d.wp = (float)w;
  d.wp64 = w;
  d.p_dyn = (float)p;
  d.p_dyn64 = p;
  d.half_dp = (float)half_dp;
  d.half_dp64 = half_dp;
  d.lpk = log2(p / kKB);
  lev[j] = d;
}

// The finite-element profile's basis at every level (Sect. 2.5.1, Eqs.
// 12-16): level j sits at x = (L - j) / L on [0,1] (x = 0 bottom), in element
// k = floor(x K_e) (clamped) at local coordinate loc = x K_e - k, where basis
// function i is prod_{m != i} (loc - xi_m) / (xi_i - xi_m).  Taken once per
// setup, so that a sample's level temperature is fe_order+1 products.
struct GllNodes {
  double v[HR2_MAX_TNODES];
};
__global__ void k_fe_basis(int n_lev, int Ke, int q, GllNodes xi, int* fe_k, double* fe_b) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n_lev) return;
  const int L = n_lev - 1;
  const double x = (double)(L - j) / (double)L;
  int k = (int)floor(x * Ke);
  k = k < 0 ? 0 : (k > Ke - 1 ? Ke - 1 : k);
  const double loc = x * Ke - k;
  for (int i = 0; i <= q; ++i) {
    double d = 1.0;
    for (int m = 0; m <= q; ++m)
      if (m != i) d *= xi.v[i] - xi.v[m];
    double l = 1.0 / d;
    for (int m = 0; m <= q; ++m)
      if (m != i) l *= loc - xi.v[m];
    fe_b[(size_t)j * (q + 1) + i] = l;
  }
  fe_k[j] = k;
}

cudaError_t build_fe_basis(int n_lev, int fe_elements, int fe_order, const double* gll, int* d_k, double* d_b,
                           cudaStream_t s) {
  GllNodes xi{};
  for (int i = 0; i <= fe_order && i < HR2_MAX_TNODES; ++i) xi.v[i] = gll[i];
  k_fe_basis<<<(n_lev + 127) / 128, 128, 0, s>>>(n_lev, fe_elements, fe_order, xi, d_k, d_b);
  return cudaGetLastError();
}

cudaError_t build_setup_levels(int n_lev, double p_top, double p_bot, const TablesDev* d_tab, LevelDev* d_levels,
                               cudaStream_t s) {
  k_levels<<<(n_lev + 127) / 128, 128, 0, s>>>(n_lev, log10(p_top), log10(p_bot), d_tab, d_levels);
  return cudaGetLastError();
}

// ------------------------------------------------ instrument profile + bins
// Gaussian instrument profile (Sect. 2.7): sigma_i = nu_i / (R 2 sqrt(2 ln 2))
// centred on output point i, kept for |nu_m - nu_i| <= 5 sigma_i and
// renormalised over the kept points.  Binning (Sect. 2.8): point i belongs to
// bin b when edge_b <= nu_i < edge_{b+1} (the last bin closed).
constexpr double kFwhmToSigma = 2.3548200450309493;  // 2 sqrt(2 ln 2)

__device__ double setup_nu(const TablesDev& t, int nu_first, int i) {
  return __dadd_rn(t.nu0, __dmul_rn((double)(nu_first + i), t.dnu));
}

__global__ void k_w_points(const TablesDev* tab, int nu_first, int n_nu, double R, int n_bins,
                           const double* __restrict__ edges, int* lo, int* hi, double* invz, int* bin) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_nu) return;
  const TablesDev& t = *tab;
  double nui = setup_nu(t, nu_first, i);
  if (R > 0.0) {
    double sig = nui / (R * kFwhmToSigma);
    double reach = 5.0 * sig;
    int k = (int)(reach / t.dnu) + 2;
    int a = max(0, i - k), b = min(n_nu - 1, i + k);
    while (a < i && fabs(setup_nu(t, nu_first, a) - nui) > reach) ++a;
    while (b > i && fabs(setup_nu(t, nu_first, b) - nui) > reach) --b;
    double z = 0.0;
    for (int m = a; m <= b; ++m) {
      double dx = setup_nu(t, nu_first, m) - nui;
      z += exp(-dx * dx / (2.0 * sig * sig));
    }
    lo[i] = a;
    hi[i] = b;
    invz[i] = 1.0 / z;
  } else {
    lo[i] = i;
    hi[i] = i;
    invz[i] = 1.0;
  }
  // bin index: -1 below the first edge, n_bins above the last one
  int bb;
  if (nui < edges[0]) {
    bb = -1;
  } else if (nui > edges[n_bins]) {
    bb = n_bins;
  } else if (nui == edges[n_bins]) {
    bb = n_bins - 1;
  } else {
    int l = 0, r = n_bins;  // largest b with edges[b] <= nui
    while (r - l > 1) {
      int mid = (l + r) / 2;
      if (edges[mid] <= nui) l = mid;
      else r = mid;
    }
    bb = l;
  }
  bin[i] = bb;
}

// rowinfo[4b..4b+3] = first member point, member count, first column, columns
__global__ void k_w_rows(int n_nu, int n_bins, const int* __restrict__ bin, const int* __restrict__ lo,
                         const int* __restrict__ hi, int* rowinfo, int* err) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= n_bins) return;
  // members of bin b form a contiguous run of the non-decreasing bin[]
  int l = 0, r = n_nu;
  while (l < r) {
    int m = (l + r) / 2;
    if (bin[m] < b) l = m + 1;
    else r = m;
  }
  int i0 = l;
  r = n_nu;
  while (l < r) {
    int m = (l + r) / 2;
    if (bin[m] <= b) l = m + 1;
    else r = m;
  }
  int cnt = l - i0;
  if (cnt <= 0) {
    atomicExch(err, 1);
    rowinfo[4 * b + 0] = 0;
    rowinfo[4 * b + 1] = 0;
    rowinfo[4 * b + 2] = 0;
    rowinfo[4 * b + 3] = 0;
    return;
  }
  int c0 = lo[i0], c1 = hi[i0];
  for (int i = i0; i < i0 + cnt; ++i) {
    c0 = min(c0, lo[i]);
    c1 = max(c1, hi[i]);
  }
  rowinfo[4 * b + 0] = i0;
  rowinfo[4 * b + 1] = cnt;
  rowinfo[4 * b + 2] = c0;
  rowinfo[4 * b + 3] = c1 - c0 + 1;
}

cudaError_t build_w_rows(const TablesDev* d_tab, int nu_first, int n_nu, double R, int n_bins,
                             const double* d_edges, int* d_lo, int* d_hi, double* d_invz, int* d_bin, int* d_rowinfo,
                             int* d_err, cudaStream_t s) {
  k_w_points<<<(n_nu + 127) / 128, 128, 0, s>>>(d_tab, nu_first, n_nu, R, n_bins, d_edges, d_lo, d_hi, d_invz, d_bin);
  k_w_rows<<<(n_bins + 127) / 128, 128, 0, s>>>(n_nu, n_bins, d_bin, d_lo, d_hi, d_rowinfo, d_err);
  return cudaGetLastError();
}

// W[b][m] = (1/n_b) sum over members i of b of g_i(m) / Z_i.
__global__ void k_w_values(const TablesDev* tab, int nu_first, double R, const int* __restrict__ lo,
                           const int* __restrict__ hi, const double* __restrict__ invz, const int* __restrict__ rowinfo,
                           const long long* __restrict__ rowptr, float* w32, double* w64) {
  int b = blockIdx.x;
  const TablesDev& t = *tab;
  int i0 = rowinfo[4 * b], cnt = rowinfo[4 * b + 1], c0 = rowinfo[4 * b + 2], nc = rowinfo[4 * b + 3];
  long long base = rowptr[b];
  for (int c = threadIdx.x; c < nc; c += blockDim.x) {
    int m = c0 + c;
    double acc = 0.0;
    if (R > 0.0) {
      double num = setup_nu(t, nu_first, m);
      for (int i = i0; i < i0 + cnt; ++i) {
        if (m < lo[i] || m > hi[i]) continue;
        double nui = setup_nu(t, nu_first, i);
        double sig = nui / (R * kFwhmToSigma);
        double dx = num - nui;
        acc += exp(-dx * dx / (2.0 * sig * sig)) * invz[i];
      }
    } else {
      acc = (m >= i0 && m < i0 + cnt) ? 1.0 : 0.0;
    }
    acc /= (double)cnt;
    w64[base + c] = acc;
    w32[base + c] = (float)acc;
  }
}

cudaError_t build_w_values(const TablesDev* d_tab, int nu_first, double R, int n_bins, const int* d_lo,
                               const int* d_hi, const double* d_invz, const int* d_rowinfo, const long long* d_rowptr,
                               float* d_w32, double* d_w64, cudaStream_t s) {
  k_w_values<<<n_bins, 256, 0, s>>>(d_tab, nu_first, R, d_lo, d_hi, d_invz, d_rowinfo, d_rowptr, d_w32, d_w64);
  return cudaGetLastError();
}

// ------------------------------------------------------- level-gridded operand
// The p part of the bilinear interpolation (Sect. 2.8), done once per setup
// in FP64 for the setup's kTileNu-point tiles t, levels j (p cell b_j,
// weight w_p), absorbers s (table species sp = species[s]) and T rows a:
//   g(a) = log2(10) ((1 - w_p) v[sp][a][b_j][col] + w_p v[sp][a][b_j+1][col])
// (log10 option) or (1 - w_p) 10^v[sp][a][b_j][col] + w_p 10^v[sp][a][b_j+1][col]
// (linear option), v the stored FP16 value log10 sigma - off_s, table column
// col = (tile0 + t) kTileNu + c; after the K absorbers come the two CIA pairs
// (which do not depend on p): h(a) = log2(10) v_cia[pair][a][col] or
// 10^v_cia[pair][a][col], zero for an absent pair.  Each is stored per T
// cell a (T rows a and a+1, n_T - 1 cells) as the row and its difference to
// row a+1, interleaved per pair of neighbouring columns:
//   lvl[t][j][a][s][q] = { g(a)[2q], g(a)[2q+1], (g(a+1)-g(a))[2q], (g(a+1)-g(a))[2q+1] }
// for s < K + 2 and q < kTileNu / 2, so that everything one level of one T
// cell needs is one contiguous block of (K + 2) x 2 kTileNu floats (one bulk
// copy), and the kernel reads a pair's value and difference with one 16-byte
// load.  The CIA rows are repeated on every level (2 of the K + 2 rows).
struct SpeciesList {
  int sp[HR2_MAX_SPECIES];
};

// row value of operand row s (absorber s < K, else CIA pair s - K) at T row a
__device__ __forceinline__ double operand_value(const TablesDev& t, const LevelDev& lv, const SpeciesList& list,
                                                int K, int s, int a, size_t col, int linear) {
  if (s < K) {
    const size_t row0 = (((size_t)list.sp[s] * t.n_T + a) * t.n_p + lv.pcell) * t.nu_pad + col;
    const double v0 = (double)__half2float(t.sig16[row0]);
    const double v1 = (double)__half2float(t.sig16[row0 + t.nu_pad]);
    return linear ? (1.0 - lv.wp64) * exp10(v0) + lv.wp64 * exp10(v1)
                  : kLog2_10 * ((1.0 - lv.wp64) * v0 + lv.wp64 * v1);
  }
  const int pair = s - K;
  if (!t.has_cia[pair]) return 0.0;
  const double v = (double)__half2float(t.cia16[((size_t)pair * t.n_T + a) * t.nu_pad + col]);
  return linear ? exp10(v) : kLog2_10 * v;
}

__global__ void k_level_cache(const TablesDev* tab, const LevelDev* lev, int n_species, SpeciesList list, int n_lev,
                              int tile0, int n_tiles, int linear, float* out) {
  const TablesDev& t = *tab;
  const int n_cells = t.n_T - 1;
  const int n_rows = n_species + 2;
  const long long total = (long long)n_tiles * n_lev * n_cells * n_rows * (2 * kTileNu);
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    long long r = idx;
    const int e = (int)(r % 4);
    r /= 4;
    const int q = (int)(r % (kTileNu / 2));
    r /= kTileNu / 2;
    const int s = (int)(r % n_rows);
    r /= n_rows;
    const int a = (int)(r % n_cells);
    r /= n_cells;
    const int j = (int)(r % n_lev);
    const int tt = (int)(r / n_lev);
    const LevelDev lv = lev[j];
    const size_t col = (size_t)(tile0 + tt) * kTileNu + 2 * q + (e & 1);
    const double g0 = operand_value(t, lv, list, n_species, s, a, col, linear);
    if (e < 2) {
      out[idx] = (float)g0;
    } else {
      const double g1 = operand_value(t, lv, list, n_species, s, a + 1, col, linear);
      out[idx] = (float)(g1 - g0);
    }
  }
}

// Wavenumber constants of the FP32 forward kernel per pair of columns.
__global__ void k_nu_pairs(const TablesDev* tab, int tile0, int n_pairs, float4* nu, float2* c1n) {
  const TablesDev& t = *tab;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n_pairs; q += gridDim.x * blockDim.x) {
    const double nu0 = t.nu0 + (double)(tile0 * kTileNu + 2 * q) * t.dnu, nu1 = nu0 + t.dnu;
    const float hi = (float)nu0;
    nu[q] = make_float4(hi, (float)(nu0 - (double)hi), (float)(nu1 / nu0), 0.f);
    c1n[q] = make_float2((float)(kC1 * nu0 * nu0 * nu0), (float)(kC1 * nu1 * nu1 * nu1));
  }
}

cudaError_t build_nu_pairs(const TablesDev* d_tab, int tile0, int n_tiles, float4* d_nu, float2* d_c1n, cudaStream_t s) {
  const int n_pairs = n_tiles * (kTileNu / 2);
  k_nu_pairs<<<(n_pairs + 255) / 256, 256, 0, s>>>(d_tab, tile0, n_pairs, d_nu, d_c1n);
  return cudaGetLastError();
}

cudaError_t build_level_cache(const TablesDev* d_tab, const SetupDev& h, float* d_lvl, cudaStream_t s) {
  SpeciesList list{};
  for (int i = 0; i < h.n_species; ++i) list.sp[i] = h.species[i];
  k_level_cache<<<4096, 256, 0, s>>>(d_tab, h.levels, h.n_species, list, h.n_lev, h.tile0, h.n_tiles,
                                     h.interp == HR2_INTERP_LINEAR, d_lvl);
  return cudaGetLastError();
}

// ------------------------------------------ streamed level-gridded operand
// The same operand as k_level_cache (layout, per tile: [level][T cell][row]
// [kTileNu/2 pairs][4]), built at evaluation time for a group of n_tiles
// consecutive tiles of setup S starting at its tile tile_lo, into ring
// (tile tt of the group at ring + tt * S.lvl32_tile_floats), in FP32
// arithmetic: g = log2(10) (v0 + w_p (v1 - v0)) of the FP16 rows v0, v1 of
// the level's p cell (log10 option only).  One thread per (tile, level, row,
// pair of columns) walks the T rows and writes each T cell's
// {g[a], g[a+1] - g[a]} of its two columns as one 16-byte store, so that 64
// threads write one cell's 1 KB block contiguously.  With a cell mask
// (this setup's [level][mask_stride] bytes, from k_mark_cells) only the cells
// some sample of the batch sits in at that level are written, from only the
// T rows they need: the sweep reads no other.
__global__ void __launch_bounds__(64) k_level_stream(const SetupDev* __restrict__ sp, int tile_lo, int n_tiles,
                                                     const unsigned char* __restrict__ mask, int mask_stride,
                                                     float* __restrict__ ring) {
  const SetupDev& S = *sp;
  const TablesDev& t = *S.tables;
  const int q = threadIdx.x;                       // pair of columns within the tile
  const int n_rows = S.n_species + 2;
  int b = blockIdx.x;
  const int s = b % n_rows;
  b /= n_rows;
  const int j = b % S.n_lev;
  const int tt = b / S.n_lev;
  if (tt >= n_tiles) return;
  const int n_cells = t.n_T - 1;
  const LevelDev lv = S.levels[j];
  const float wp = (float)lv.wp64;
  const float l2 = (float)kLog2_10;
  const size_t col = (size_t)(S.tile0 + tile_lo + tt) * kTileNu + 2 * q;
  const __half* base;
  size_t a_step;
  bool interp = true, zero = false;
  if (s < S.n_species) {
    base = t.sig16 + (((size_t)S.species[s] * t.n_T) * t.n_p + lv.pcell) * t.nu_pad + col;
    a_step = (size_t)t.n_p * t.nu_pad;
  } else {
    const int pair = s - S.n_species;
    base = t.cia16 + (size_t)pair * t.n_T * t.nu_pad + col;
    a_step = (size_t)t.nu_pad;
    interp = false;
    zero = !t.has_cia[pair];
  }
  float4* out = reinterpret_cast<float4*>(ring + (size_t)tt * S.lvl32_tile_floats) +
                (((size_t)j * n_cells) * n_rows + s) * (kTileNu / 2) + q;
  const size_t cell_step = (size_t)n_rows * (kTileNu / 2);   // float4s from one T cell to the next
  const unsigned char* mrow = mask ? mask + (size_t)j * mask_stride : nullptr;
  float2 gp = make_float2(0.f, 0.f);
  for (int a = 0; a < t.n_T; ++a) {
    float2 g = make_float2(0.f, 0.f);
    // T row a enters the cells a-1 and a; with a mask it is read only if one of them is built
    const bool need = !mrow || (a > 0 && mrow[a - 1]) || (a < n_cells && mrow[a]);
    if (!zero && need) {
      const __half2 h0 = *reinterpret_cast<const __half2*>(base + a * a_step);
      const float2 v0 = __half22float2(h0);
      if (interp) {
        const float2 v1 = __half22float2(*reinterpret_cast<const __half2*>(base + a * a_step + t.nu_pad));
        g = make_float2(l2 * fmaf(wp, v1.x - v0.x, v0.x), l2 * fmaf(wp, v1.y - v0.y, v0.y));
      } else {
        g = make_float2(l2 * v0.x, l2 * v0.y);
      }
    }
    if (a > 0 && (!mrow || mrow[a - 1]))
      out[(size_t)(a - 1) * cell_step] = make_float4(gp.x, gp.y, g.x - gp.x, g.y - gp.y);
    gp = g;
  }
}

// The T cells the batch's valid samples sit in, per setup and level:
// mask[(g * max_lev + j) * stride + a] = 1 where some sample of setup g has
// cell a in its record of level j (records of the level-gridded sweep,
// written by k_prep).  The mask starts at zero.
__global__ void k_mark_cells(FwdArgs a, int max_lev, int stride, unsigned char* mask) {
  const long long total = (long long)a.n * max_lev;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(idx / max_lev), j = (int)(idx % max_lev);
    const SampleDev& sd = a.samp[i];
    if (sd.status != 0 || sd.setup < 0 || sd.setup >= a.n_setups) continue;
    const SetupDev& S = *a.setups[sd.setup];
    if (j >= S.n_lev) continue;
    const int c = reinterpret_cast<const LevRecC*>(a.recs + (size_t)i * a.rec_ld)[j].acell;
    if (c >= 0 && c < S.tables->n_T - 1 && c < stride) mask[((size_t)sd.setup * max_lev + j) * stride + c] = 1;
  }
}

cudaError_t build_cell_mask(const FwdArgs& a, int max_lev, int stride, unsigned char* mask, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(mask, 0, (size_t)a.n_setups * max_lev * stride, s);
  if (e != cudaSuccess || a.n <= 0) return e;
  const long long total = (long long)a.n * max_lev;
  const int blocks = (int)std::min<long long>((total + 255) / 256, 4096);
  k_mark_cells<<<blocks, 256, 0, s>>>(a, max_lev, stride, mask);
  return cudaGetLastError();
}

// One setup view per group of group_tiles tiles, for setup `ord` of a batch
// of n_setups (views[g * n_setups + ord]): the setup with its tile range,
// wavenumber constants and operand narrowed to the group and the operand
// read from its section of the ring (the forward kernel then sees an
// ordinary level-gridded setup of up to group_tiles tiles, none once the
// setup's tiles are all behind; its output columns stay those of the whole
// setup, since they follow tile0 and nu_first).
__global__ void k_stream_views(const SetupDev* __restrict__ sp, const float* ring, int group_tiles, int n_groups,
                               int ord, int n_setups, SetupDev* views) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n_groups) return;
  SetupDev v = *sp;
  const int lo = min(g * group_tiles, sp->n_tiles);
  v.tile0 = sp->tile0 + lo;
  v.n_tiles = min(group_tiles, sp->n_tiles - lo);
  v.nu_pair = sp->nu_pair + (size_t)lo * (kTileNu / 2);
  v.c1n_pair = sp->c1n_pair + (size_t)lo * (kTileNu / 2);
  v.lvl32 = ring;
  v.cached = 1;
  views[(size_t)g * n_setups + ord] = v;
}

cudaError_t build_level_stream(const SetupDev* d_setup, int n_lev, int n_rows, int tile_lo, int n_tiles,
                               const unsigned char* mask, int mask_stride, float* ring, cudaStream_t s) {
  const long long blocks = (long long)n_tiles * n_lev * n_rows;
  if (blocks <= 0) return cudaSuccess;
  if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
  k_level_stream<<<(unsigned)blocks, kTileNu / 2, 0, s>>>(d_setup, tile_lo, n_tiles, mask, mask_stride, ring);
  return cudaGetLastError();
}

cudaError_t build_stream_views(const SetupDev* d_setup, const float* ring, int group_tiles, int n_groups, int ord,
                               int n_setups, SetupDev* views, cudaStream_t s) {
  if (n_groups <= 0) return cudaSuccess;
  k_stream_views<<<(n_groups + 127) / 128, 128, 0, s>>>(d_setup, ring, group_tiles, n_groups, ord, n_setups, views);
  return cudaGetLastError();
}

}  // namespace hr2
