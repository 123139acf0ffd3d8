// kern_forward.cu -- the per-batch kernels of the forward model:
//   k_prep       per (sample, level): T profile, interpolation cells and
//                weights, CIA and Planck factors (FP64 math, FP32 records)
//   k_plan       groups samples by setup and lays out the work items
//   k_forward32  persistent FP32 kernel over (setup, wavenumber tile,
//                sample block) items: opacity interpolation, absorption,
//                optical depth, Planck source, short characteristics,
//                angular quadrature -> F+
//   k_forward64  the plain FP64 path: same steps in double, one thread per
//                wavenumber, FP64 tables
//   k_bins       instrument profile + binning via the setup's operator W
//   k_lnl        Gaussian log-likelihood, FP64, fixed-order warp reduction
#include <math.h>
#include <stddef.h>

#include "hr2_internal.cuh"
#include "kern_forward32.cuh"

namespace hr2 {
// Continuous finite-element temperature at x in [0,1] (x = 0 bottom, 1 top):
// element k of K_e, local coordinate on [0,1] with the Gauss-Lobatto nodes,
// Lagrange basis (Sect. 2.5.1, Eqs. 12-16).  Node 0 is the bottom T_1.
__device__ double fe_temperature(const SetupDev& S, const double* nodes, double x) {
  const int Ke = S.fe_elements, q = S.fe_order;
  int k = (int)floor(x * Ke);
  k = k < 0 ? 0 : (k > Ke - 1 ? Ke - 1 : k);
  const double loc = x * Ke - k;
  double T = 0.0;
  for (int i = 0; i <= q; ++i) {
    double l = 1.0;
    for (int m = 0; m <= q; ++m)
      if (m != i) l *= (loc - S.gll[m]) / (S.gll[i] - S.gll[m]);
    T += nodes[k * q + i] * l;
  }
  return T;
}

// The same profile at level j from the setup's basis values there (element
// fe_k[j], basis fe_b[j][i]): fe_order+1 products per level.
__device__ __forceinline__ double fe_temperature_level(const SetupDev& S, const double* nodes, int j) {
  const int q = S.fe_order, k = S.fe_k[j];
  const double* b = S.fe_b + (size_t)j * (q + 1);
  double T = 0.0;
  for (int i = 0; i <= q; ++i) T += nodes[k * q + i] * b[i];
  return T;
}

// 2^b for the FP32 record fields: 2^rint(b) exactly times exp2f of the
// remainder (|r| <= 1/2, relative error ~2e-7), without FP64 transcendentals.
__device__ __forceinline__ float exp2_split(double b) {
  const double n = rint(b);
  return ldexpf(exp2f((float)(b - n)), (int)n);
}

// Hopf function q(tau) from the setup's table: cubic Lagrange interpolation in
// ln tau through the four nearest nodes (the stencil slides inward at the
// table's ends); q(kHopfTau0) below the table, q(kHopfTau1) above it.
__device__ double hopf_q(const double* tab, double tau) {
  if (!(tau > kHopfTau0)) return tab[0];
  const double u = (log(tau) - log(kHopfTau0)) * ((kHopfN - 1) / (log(kHopfTau1) - log(kHopfTau0)));
  if (!(u < kHopfN - 1)) return tab[kHopfN - 1];
  const int k0 = min(max((int)u - 1, 0), kHopfN - 4);
  const double x = u - (double)k0;              // in [0, 3]: nodes at 0, 1, 2, 3
  const double a = x - 1.0, b = x - 2.0, c = x - 3.0;
  return (-a * b * c * tab[k0] + 3.0 * x * b * c * tab[k0 + 1] - 3.0 * x * a * c * tab[k0 + 2] +
          x * a * b * tab[k0 + 3]) * (1.0 / 6.0);
}

// Temperature of level j (0 = top) of sample parameters th (Sect. 2.5): the
// finite-element profile, or Milne's T^4 = 3/4 Tbar^4 (tau_R + q(tau_R)) with
// tau_R = kappa_R p_j / g (th[3] = Tbar in K, th[4] = log10 kappa_R in cm^2/g).
__device__ double level_temperature(const SetupDev& S, const double* th, int j, double grav) {
  const int L = S.n_lev - 1;
  if (S.profile == HR2_PROFILE_MILNE) {
    const double tau = exp10(th[HR2_P_T0 + 1]) * S.levels[j].p_dyn64 / grav;
    const double tb = th[HR2_P_T0];
    return pow(0.75 * tb * tb * tb * tb * (tau + hopf_q(S.hopf_q, tau)), 0.25);
  }
  return fe_temperature(S, th + HR2_P_T0, (double)(L - j) / (double)L);
}

// Cell a with grid[a] <= v <= grid[a+1] and the weight of grid[a+1],
// clamped to the grid ends (no extrapolation).
__device__ void grid_cell(const double* grid, int n, double v, int& a, double& w) {
  if (!(v > grid[0])) {
    a = 0;
    w = 0.0;
    return;
  }
  if (v >= grid[n - 1]) {
    a = n - 2;
    w = 1.0;
    return;
  }
  int lo = 0, hi = n - 1;
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (grid[mid] < v) lo = mid;
    else hi = mid;
  }
  a = lo;
  w = (v - grid[lo]) / (grid[lo + 1] - grid[lo]);
}

// added to every layer's optical depth on the linear-source path (in the
// level record), so that dtau > 0 and (S_j - S_{j-1}) / dtau stays finite in
// an opacity-free layer (|S| < 3e18); a layer this thin is transparent either
// way (its factor (1 - e^{-D}) / dtau is 1/mu to FP32 precision below
// dtau ~ 1e-8)
constexpr float kTinyTau = 1e-20f;

// ------------------------------------------------------------------ prep
// One warp per sample.  Free chemistry (Sect. 2.4): absorber mixing ratios
// x_s, H2 and He fill the rest at n_He/n_H2 = r_he; the column factor
// c = 1/(mmw m_u g) turns a cross-section per molecule into optical depth
// per unit pressure (hydrostatic dm = dp/g).
__global__ void k_prep(FwdArgs a) {
  const int lane = threadIdx.x & 31;
  const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (i >= a.n) return;
  SampleDev* sd = a.samp + i;
  const int g = a.setup_of_sample[i];
  if (g < 0 || g >= a.n_setups) {
    if (lane == 0) {
      sd->status = HR2_SAMPLE_BAD_SETUP;
      sd->setup = -1;
      sd->scale = 0.0;
      sd->scale32[0] = sd->scale32[1] = 0.f;
      if (a.status) a.status[i] = HR2_SAMPLE_BAD_SETUP;
    }
    return;
  }
  const SetupDev& S = *a.setups[g];
  const TablesDev& T = *S.tables;
  if constexpr (HR2_BOUNDS_CHECK) {
    // the sample's record row and the setup's species and level cells
    bool ok = S.n_lev <= a.rec_ld && S.n_species <= HR2_MAX_SPECIES && S.n_species <= T.n_species;
    for (int s = 0; s < S.n_species; ++s) ok = ok && S.species[s] >= 0 && S.species[s] < T.n_species;
    for (int j = lane; ok && j < S.n_lev; j += 32) ok = S.levels[j].pcell >= 0 && S.levels[j].pcell <= T.n_p - 2;
    if (!bounds_ok(__all_sync(0xffffffffu, ok), lane == 0 ? a.err : nullptr)) {
      if (lane == 0) {
        sd->status = HR2_SAMPLE_BAD_SETUP;
        sd->setup = -1;
        if (a.status) a.status[i] = HR2_SAMPLE_BAD_SETUP;
      }
      return;
    }
  }
  const double* th = a.params + (size_t)i * HR2_NPARAM;
  const unsigned full = 0xffffffffu;
  int status = 0;
  // The sample's scalar transcendentals, one per lane so that the warp
  // evaluates them in one pass of its FP64 units: lane s < K 10^(log10 x_s),
  // lane kLaneG 10^(log10 g), lanes kLaneC.. the cloud's three powers of 10.
  constexpr int kLaneG = HR2_MAX_SPECIES, kLaneC = HR2_MAX_SPECIES + 1;
  double e10 = 0.0;
  {
    double arg = 0.0;
    if (lane < S.n_species) {
      arg = th[HR2_P_X0 + lane];
      if (!isfinite(arg)) status |= HR2_SAMPLE_BAD_ABUND;
    } else if (lane == kLaneG) {
      arg = th[HR2_P_LOGG];
    } else if (S.cloud && lane >= kLaneC && lane < kLaneC + 3) {
      arg = th[HR2_P_CLOUD + (lane - kLaneC)];
    }
    e10 = exp10(arg);
  }
  // sums in species order
  double sumx = 0.0, mabs = 0.0;
  for (int s = 0; s < S.n_species; ++s) {
    const double x = __shfl_sync(full, e10, s);
    sumx += x;
    mabs += x * S.mass64[s];
  }
  if (!(sumx < 1.0)) status |= HR2_SAMPLE_BAD_ABUND;
  const double xh2 = (1.0 - sumx) / (1.0 + S.r_he);
  const double xhe = S.r_he * xh2;
  const double mmw = mabs + xh2 * kMassH2 + xhe * kMassHe;
  const double grav = __shfl_sync(full, e10, kLaneG);
  const double f = th[HR2_P_F], dcm = th[HR2_P_DIST] * kParsec;
  if (!(f > 0.0) || !(dcm > 0.0) || !isfinite(f) || !isfinite(dcm) || !isfinite(grav) || !(grav > 0.0))
    status |= HR2_SAMPLE_BAD_SCALE;
  const double c = 1.0 / (mmw * kAMU * grav);
  // log2 of c, x_H2 and x_He, one per lane
  const double l2 = log2(lane == 0 ? c : (lane == 1 ? xh2 : xhe));
  const double lc = __shfl_sync(full, l2, 0);
  const double ratio = S.radius_cm / dcm;
  // integer shift that centres the exponent of the dominant absorber
  double amax = -1e300;
  for (int s = 0; s < S.n_species; ++s)
    amax = fmax(amax, th[HR2_P_X0 + s] * kLog2_10 + lc + T.off[S.species[s]] * kLog2_10);
  const double shift = (S.n_species > 0 && isfinite(amax)) ? rint(amax) : 0.0;
  if (lane < S.n_species) {
    const double A = th[HR2_P_X0 + lane] * kLog2_10 + lc + T.off[S.species[lane]] * kLog2_10 - shift;
    const float hi = (float)A;
    sd->A[lane] = hi;
    sd->Ac[lane] = (float)(1.0 + kLn2 * (A - (double)hi));
    sd->W[lane] = (float)exp2(A);
  }

  // gray cloud layer: tau_c spread evenly in pressure over [pct, pcb]
  double tau_c = 0.0, pct = 0.0, pcb = 0.0;
  if (S.cloud) {
    tau_c = __shfl_sync(full, e10, kLaneC);
    pct = __shfl_sync(full, e10, kLaneC + 1) * kBar;
    const double fc = __shfl_sync(full, e10, kLaneC + 2);
    if (!isfinite(tau_c) || !(tau_c >= 0.0) || !(pct > 0.0) || !isfinite(pct) || !(fc > 0.0) || !(fc <= 1.0))
      status |= HR2_SAMPLE_BAD_CLOUD;
    pcb = pct / fc;
  }

  const int L = S.n_lev - 1;
  LevRec* rec = a.recs + (size_t)i * a.rec_ld;
  // per-sample constants of the level records: log2 of the CIA prefactors
  // without the level's number density, b = log2(x x' c n_j) + off log2 10 -
  // shift = cb + log2(p_j / k_B) - log2 T_j
  const double lxh2 = __shfl_sync(full, l2, 1), lxhe = __shfl_sync(full, l2, 2);
  const double cb0 = 2.0 * lxh2 + lc + T.off[kCiaH2H2] * kLog2_10 - shift;
  const double cb1 = lxh2 + lxhe + lc + T.off[kCiaH2He] * kLog2_10 - shift;
  const float tiny = (S.sc != HR2_SC_PARABOLIC) ? kTinyTau : 0.f;
  for (int j = lane; j <= L; j += 32) {
    const double Tj = S.profile == HR2_PROFILE_MILNE
                          ? level_temperature(S, th, j, grav)
                          : fe_temperature_level(S, th + HR2_P_T0, j);
    if (!(Tj > 0.0) || !isfinite(Tj)) status |= HR2_SAMPLE_BAD_T;
    int acell;
    double wT;
    grid_cell(T.T_grid64, T.n_T, Tj, acell, wT);
    if constexpr (HR2_BOUNDS_CHECK) {
      if (!bounds_ok(acell >= 0 && acell <= T.n_T - 2, a.err)) acell = 0;
    }
    const LevelDev lv = S.levels[j];
    const double lT = log2(Tj);
    const double b0 = cb0 + lv.lpk - lT;    // log2(x_H2^2 c n_j) + off log2 10 - shift
    const double b1 = cb1 + lv.lpk - lT;    // log2(x_H2 x_He c n_j) + off log2 10 - shift
    const double upl = kC2 * kLog2e / Tj;   // e^{hc nu/kT} = 2^(upl nu)
    const float half_dp = (float)ldexp(lv.half_dp64, (int)shift);
    const float rnu = exp2f((float)(upl * T.dnu));           // e^{hc dnu/kT}, argument << 1
    const float r64 = exp2f((float)(upl * T.dnu * kPairStride));   // e^{64 hc dnu/kT}
    // zero for an absent pair: the cached path adds both pairs unconditionally
    const float wh2h2 = T.has_cia[0] ? exp2_split(b0) : 0.f;
    const float wh2he = T.has_cia[1] ? exp2_split(b1) : 0.f;
    float dtc = 0.f;
    if (S.cloud && j > 0 && pcb > pct) {   // layer j-1 between levels j-1 and j
      const double lo = fmax(S.levels[j - 1].p_dyn64, pct), hi = fmin(lv.p_dyn64, pcb);
      if (hi > lo) dtc = (float)(tau_c * (hi - lo) / (pcb - pct));
    }
    dtc += tiny;
    if (S.cached) {
      LevRecC rc;
      rc.wT[0] = rc.wT[1] = (float)wT;
      rc.wh2h2[0] = rc.wh2h2[1] = wh2h2;
      rc.wh2he[0] = rc.wh2he[1] = wh2he;
      rc.half_dp[0] = rc.half_dp[1] = half_dp;
      rc.dtc[0] = rc.dtc[1] = dtc;
      rc.upl = (float)upl;
      rc.rnu = rnu;
      rc.acell = acell;
      // the level's operand block of T cell acell within a tile
      rc.lvl_off = (j * (T.n_T - 1) + acell) * (S.n_species + 2) * 2 * kTileNu;
      rc.r64 = r64;
      rc.pad = 0;
      reinterpret_cast<LevRecC*>(rec)[j] = rc;
    } else {
      const double wp = lv.wp64;
      LevRec r;
      r.rowoff = acell * T.n_p + lv.pcell;
      r.acell = acell;
      r.wT = (float)wT;
      r.wp = (float)wp;
      r.wTwp = (float)(wT * wp);
      r.bh2h2 = (float)b0;
      r.ch2h2 = (float)(1.0 + kLn2 * (b0 - (double)r.bh2h2));
      r.bh2he = (float)b1;
      r.ch2he = (float)(1.0 + kLn2 * (b1 - (double)r.bh2he));
      r.upl = (float)upl;
      r.r64 = r64;
      r.half_dp = half_dp;
      r.rnu = rnu;
      r.wh2h2 = wh2h2;
      r.wh2he = wh2he;
      r.dtau_cloud = dtc;
      rec[j] = r;
    }
  }
  status = __reduce_or_sync(0xffffffffu, status);
  if (lane == 0) {
    sd->status = status;
    const double sc = f * ratio * ratio;
    sd->scale = sc;
    sd->scale32[0] = (float)sc;
    sd->scale32[1] = (float)(sc - (double)(float)sc);
    sd->setup = g;
    if (a.status) a.status[i] = status;
  }
}

cudaError_t launch_prep(const FwdArgs& a, cudaStream_t s) {
  if (a.n <= 0) return cudaSuccess;
  // one warp per sample, two per block: a 1024-sample batch spreads over
  // every SM (the per-level work is FP64)
  k_prep<<<(a.n + 1) / 2, 64, 0, s>>>(a);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ plan
// Counts samples per setup, orders setups by decreasing item cost, lays out
// work items (setup, group of tiles_per_item consecutive tiles, sample block)
// with the sample block fastest so that consecutive items share wavenumber
// tiles of the table, and writes the samples of each setup contiguously
// (stable) into perm.
__global__ void k_plan(FwdArgs a, int* perm, PlanDev* plan) {
  __shared__ int cnt[HR2_MAX_SETUPS], base[HR2_MAX_SETUPS];
  const int tid = threadIdx.x;
  if (tid < HR2_MAX_SETUPS) cnt[tid] = 0;
  __syncthreads();
  for (int i = tid; i < a.n; i += blockDim.x) {
    const int g = a.setup_of_sample[i];
    if (g >= 0 && g < a.n_setups) atomicAdd(&cnt[g], 1);
  }
  __syncthreads();
  if (tid == 0) {
    int order[HR2_MAX_SETUPS];
    for (int g = 0; g < a.n_setups; ++g) order[g] = g;
    for (int p = 1; p < a.n_setups; ++p) {  // stable insertion sort, cost descending
      int v = order[p], q = p - 1;
      while (q >= 0 && a.setups[order[q]]->cost < a.setups[v]->cost) {
        order[q + 1] = order[q];
        --q;
      }
      order[q + 1] = v;
    }
    int first = 0;
    for (int g = 0; g < a.n_setups; ++g) {
      plan->first[g] = first;
      base[g] = first;
      plan->count[g] = cnt[g];
      plan->n_sblocks[g] = (cnt[g] + a.warps - 1) / a.warps;
      first += cnt[g];
    }
    int items = 0;
    for (int p = 0; p < a.n_setups; ++p) {
      const int g = order[p];
      plan->order[p] = g;
      plan->item_start[p] = items;
      const int tpi = a.tiles_per_item > 0 ? a.tiles_per_item : 1;
      items += plan->n_sblocks[g] * ((a.setups[g]->n_tiles + tpi - 1) / tpi);
    }
    plan->item_start[a.n_setups] = items;
    plan->total_items = items;
    plan->n_setups = a.n_setups;
    *a.counter = 0u;
    if (a.err) *a.err = 0;
  }
  __syncthreads();
  if (tid < 32) {
    const int lane = tid;
    for (int c0 = 0; c0 < a.n; c0 += 32) {
      const int i = c0 + lane;
      const int g = (i < a.n) ? a.setup_of_sample[i] : -1;
      const bool ok = g >= 0 && g < a.n_setups;
      const int key = ok ? g : -1;
      const unsigned peers = __match_any_sync(0xffffffffu, key);
      const int rank = __popc(peers & ((1u << lane) - 1u));
      const int leader = __ffs(peers) - 1;
      const int b = ok ? base[g] : 0;
      __syncwarp();
      if (ok) perm[b + rank] = i;
      if (ok && lane == leader) base[g] = b + __popc(peers);
      __syncwarp();
    }
  }
}

cudaError_t launch_plan(const FwdArgs& a, int* perm, PlanDev* plan, cudaStream_t s) {
  k_plan<<<1, 1024, 0, s>>>(a, perm, plan);
  return cudaGetLastError();
}

size_t forward32_smem_bytes(int warps, int max_k, int stages) { return (size_t)warps * warp_pipe_bytes(max_k, stages); }

// ------------------------------------------------------- two-pass direct path
// First pass for small batches on FP16 tables read in place: every level's
// absorption coefficient chi, for all levels and tiles of a sample at once
// (one warp per (sample, level, tile): far more warps than one per tile have
// table reads in flight), with the sweep's own arithmetic (direct_level_chi),
// so that the second pass -- the level sweep reading chi back -- gives the
// one-pass result bit for bit.  A CTA holds four consecutive levels of one
// sample and tile, and the tile is the grid's fastest index: the CTAs in
// flight at one time take neighbouring tiles of the same levels, so they
// read the same table rows (few distinct pages) at neighbouring columns.
__global__ void __launch_bounds__(128) k_chi_direct(FwdArgs a) {
  __shared__ const void* sPtr[HR2_MAX_SPECIES];
  __shared__ v2 sA2[HR2_MAX_SPECIES], sAc2[HR2_MAX_SPECIES];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int i = blockIdx.z, tile = blockIdx.x, j = blockIdx.y * 4 + warp;
  const SampleDev& sd = a.samp[i];
  const int g = sd.setup;
  if (g < 0 || g >= a.n_setups || sd.status != 0) return;   // the same for the whole CTA
  const SetupDev& S = *a.setups[g];
  if (tile >= S.n_tiles) return;
  const TablesDev& T = *S.tables;
  if (threadIdx.x < S.n_species) {
    sPtr[threadIdx.x] = T.sig16 + (size_t)S.species[threadIdx.x] * T.n_T * T.n_p * T.nu_pad;
    sA2[threadIdx.x] = pk(sd.A[threadIdx.x]);
    sAc2[threadIdx.x] = pk(sd.Ac[threadIdx.x]);
  }
  __syncthreads();
  if (j >= S.n_lev) return;
  const LevRec* rec = a.recs + (size_t)i * a.rec_ld;
  if constexpr (HR2_BOUNDS_CHECK) {
    const LevRec r = rec[j];
    bool ok = S.n_lev <= a.rec_ld && (long long)(tile + 1) * kTileNu <= a.chi_ld &&
              (long long)(S.tile0 + tile + 1) * kTileNu <= T.nu_pad && r.acell >= 0 && r.acell <= T.n_T - 2 &&
              r.rowoff >= 0 && r.rowoff / T.n_p == r.acell && r.rowoff % T.n_p <= T.n_p - 2;
    for (int s = 0; s < S.n_species; ++s) ok = ok && S.species[s] >= 0 && S.species[s] < T.n_species;
    if (!bounds_ok(ok, lane == 0 ? a.err : nullptr)) return;
  }
  const float4* q = reinterpret_cast<const float4*>(rec) + 4 * j;
  const float4 r0 = __ldg(q), r1 = __ldg(q + 1), r2 = __ldg(q + 2);
  const int col = (S.tile0 + tile) * kTileNu + 2 * lane;
  v2 chi[kPairs];
  direct_level_chi(T, S.n_species, col, r0, r1, r2, sA2, sAc2, sPtr, T.has_cia[0] != 0, T.has_cia[1] != 0, chi);
  float* out = a.chi + ((size_t)i * a.rec_ld + j) * a.chi_ld + (size_t)tile * kTileNu + 2 * lane;
#pragma unroll
  for (int p = 0; p < kPairs; ++p) *reinterpret_cast<v2*>(out + 64 * p) = chi[p];
}

cudaError_t launch_chi_direct(const FwdArgs& a, int max_lev, int max_tiles, cudaStream_t s) {
  if (a.n <= 0) return cudaSuccess;
  const dim3 grid(max_tiles, (max_lev + 3) / 4, a.n);
  k_chi_direct<<<grid, 128, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_forward32(const FwdArgs& a, int max_nmu, int grid, bool cached, bool linear, bool para, int max_k,
                             int kt, int stages, cudaStream_t s) {
  switch (max_nmu) {
    case 1: return launch_forward32_n1(a, grid, cached, linear, para, max_k, kt, stages, s);
    case 2: return launch_forward32_n2(a, grid, cached, linear, para, max_k, kt, stages, s);
    case 3: return launch_forward32_n3(a, grid, cached, linear, para, max_k, kt, stages, s);
    case 4: return launch_forward32_n4(a, grid, cached, linear, para, max_k, kt, stages, s);
    case 5: return launch_forward32_n5(a, grid, cached, linear, para, max_k, kt, stages, s);
    case 6: return launch_forward32_n6(a, grid, cached, linear, para, max_k, kt, stages, s);
    case 7: return launch_forward32_n7(a, grid, cached, linear, para, max_k, kt, stages, s);
    case 8: return launch_forward32_n8(a, grid, cached, linear, para, max_k, kt, stages, s);
    default: return cudaErrorInvalidValue;
  }
}

// ---------------------------------------------------- effective temperature
// T_eff per sample (Sect. 2.6): F+ (the library's high-resolution output,
// before the distance dilution) integrated over the sample's setup grid by
// the trapezoid rule in FP64 (lane-strided sums, fixed-order butterfly), then
// F = sigma T_eff^4.  One warp per sample.
__global__ void k_teff(FwdArgs a, const float* __restrict__ highres, int ld, double* out) {
  const int lane = threadIdx.x & 31;
  const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (i >= a.n) return;
  const int g = a.setup_of_sample[i];
  if (g < 0 || g >= a.n_setups) {
    if (lane == 0) out[i] = __longlong_as_double(0x7ff8000000000000ll);
    return;
  }
  const SetupDev& S = *a.setups[g];
  const float* F = highres + (size_t)i * ld;
  const int n = S.n_nu;
  double acc = 0.0;
  for (int k = lane; k < n; k += 32) acc += (double)F[k];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) {
    const double trap = S.tables->dnu * (acc - 0.5 * ((double)F[0] + (double)F[n - 1]));
    out[i] = pow(trap / kSigmaSB, 0.25);
  }
}

cudaError_t launch_teff(const FwdArgs& a, const float* highres, int highres_ld, double* out, cudaStream_t s) {
  if (a.n <= 0) return cudaSuccess;
  k_teff<<<(a.n + 7) / 8, 256, 0, s>>>(a, highres, highres_ld, out);
  return cudaGetLastError();
}

// ---------------------------------------------------------- FP64 forward
// M_k(D) = int_0^D t^k e^{-t} dt for k = 0, 1, 2: power series
// sum_n (-1)^n D^{k+n+1} / (n! (k+n+1)) below D = 1/2, closed forms
// (1 - e^{-D}, M_0 - D e^{-D}, 2 M_1 - D^2 e^{-D}) above.
__device__ void exp_moments(double D, double& M0, double& M1, double& M2) {
  if (D < 0.5) {
    double term = D, s0 = 0.0, s1 = 0.0, s2 = 0.0;   // term = (-1)^n D^{n+1} / n!
    for (int n = 0; n < 40; ++n) {
      s0 += term / (n + 1);
      s1 += term * D / (n + 2);
      s2 += term * D * D / (n + 3);
      term *= -D / (n + 1);
      if (fabs(term) < 1e-30) break;
    }
    M0 = s0;
    M1 = s1;
    M2 = s2;
  } else {
    const double e = exp(-D);
    M0 = -expm1(-D);
    M1 = M0 - D * e;
    M2 = 2.0 * M1 - D * D * e;
  }
}

// The plain FP64 path: one thread per wavenumber point, one block per
// (sample, 128-point chunk), FP64 tables, exp/expm1 in double.
constexpr int kF64Block = 128;

template <int NMU>
__global__ void __launch_bounds__(kF64Block) k_forward64(FwdArgs a) {
  __shared__ double sT[HR2_MAX_LEVELS], sN[HR2_MAX_LEVELS], swT[HR2_MAX_LEVELS];
  __shared__ int sa[HR2_MAX_LEVELS];
  __shared__ double sx[HR2_MAX_SPECIES];
  __shared__ double sc[6];
  const int i = blockIdx.y;
  const SampleDev& sd = a.samp[i];
  if (sd.setup < 0) return;
  const SetupDev& S = *a.setups[sd.setup];
  const TablesDev& T = *S.tables;
  if (blockIdx.x * kF64Block >= S.n_nu) return;
  const int k = blockIdx.x * kF64Block + threadIdx.x;
  double* out = a.highres64 + (size_t)i * a.highres64_ld;
  float* uout = a.user_highres ? a.user_highres + (size_t)i * a.highres_ld : nullptr;
  if (sd.status != 0) {
    if (k < S.n_nu) {
      out[k] = __longlong_as_double(0x7ff8000000000000ll);
      if (uout) uout[k] = __int_as_float(0x7fc00000);
    }
    return;
  }
  const double* th = a.params + (size_t)i * HR2_NPARAM;
  if (threadIdx.x < S.n_species) sx[threadIdx.x] = exp10(th[HR2_P_X0 + threadIdx.x]);
  __syncthreads();
  if (threadIdx.x == 0) {
    double sumx = 0.0, mabs = 0.0;
    for (int s = 0; s < S.n_species; ++s) {
      sumx += sx[s];
      mabs += sx[s] * S.mass64[s];
    }
    const double xh2 = (1.0 - sumx) / (1.0 + S.r_he);
    const double xhe = S.r_he * xh2;
    const double mmw = mabs + xh2 * kMassH2 + xhe * kMassHe;
    sc[0] = 1.0 / (mmw * kAMU * exp10(th[HR2_P_LOGG]));
    sc[1] = xh2;
    sc[2] = xhe;
    sc[3] = sc[4] = sc[5] = 0.0;   // gray cloud: tau_c, top and bottom pressure
    if (S.cloud) {
      sc[3] = exp10(th[HR2_P_CLOUD]);
      sc[4] = exp10(th[HR2_P_CLOUD + 1]) * kBar;
      sc[5] = sc[4] / exp10(th[HR2_P_CLOUD + 2]);
    }
  }
  const int L = S.n_lev - 1;
  const double grav = exp10(th[HR2_P_LOGG]);
  for (int j = threadIdx.x; j <= L; j += kF64Block) {
    const double Tj = level_temperature(S, th, j, grav);
    int ac;
    double w;
    grid_cell(T.T_grid64, T.n_T, Tj, ac, w);
    sT[j] = Tj;
    sa[j] = ac;
    swT[j] = w;
    sN[j] = S.levels[j].p_dyn64 / (kKB * Tj);
  }
  __syncthreads();
  if (k >= S.n_nu) return;
  const double c = sc[0], xh2 = sc[1], xhe = sc[2];
  const int col = S.nu_first + k;
  const double nu = T.nu0 + (double)col * T.dnu;
  const int nu_pad = T.nu_pad, np = T.n_p;
  const bool lin = S.interp == HR2_INTERP_LINEAR;   // interpolation space of the tables
  const bool para = S.sc == HR2_SC_PARABOLIC;
  // chi and S of level jj
  auto level = [&](int jj, double& chi, double& Sv) {
    const LevelDev& lv = S.levels[jj];
    const double wT = swT[jj], wp = lv.wp64;
    const size_t row = ((size_t)sa[jj] * np + lv.pcell) * nu_pad + col;
    chi = 0.0;
    for (int s = 0; s < S.n_species; ++s) {
      const double* t = T.sig64 + (size_t)S.species[s] * T.n_T * np * nu_pad + row;
      const double* t10 = t + (size_t)np * nu_pad;
      const double sig = lin ? (1.0 - wT) * (1.0 - wp) * exp10(t[0]) + wT * (1.0 - wp) * exp10(t10[0]) +
                                   (1.0 - wT) * wp * exp10(t[nu_pad]) + wT * wp * exp10(t10[nu_pad])
                             : exp10((1.0 - wT) * (1.0 - wp) * t[0] + wT * (1.0 - wp) * t10[0] +
                                     (1.0 - wT) * wp * t[nu_pad] + wT * wp * t10[nu_pad]);
      chi += sx[s] * sig;
    }
    for (int p = 0; p < 2; ++p) {
      if (!T.has_cia[p]) continue;
      const double* t = T.cia64 + (size_t)p * T.n_T * nu_pad + (size_t)sa[jj] * nu_pad + col;
      const double kcia =
          lin ? (1.0 - wT) * exp10(t[0]) + wT * exp10(t[nu_pad]) : exp10((1.0 - wT) * t[0] + wT * t[nu_pad]);
      chi += xh2 * (p == 0 ? xh2 : xhe) * sN[jj] * kcia;
    }
    Sv = kC1 * nu * nu * nu / expm1(kC2 * nu / sT[jj]);
  };
  // optical depth of layer jj (levels jj, jj+1): trapezoid of chi plus the gray cloud's share
  auto layer_dtau = [&](int jj, double chi_top, double chi_bot) {
    const LevelDev& lv = S.levels[jj];
    double dtau = (chi_top + chi_bot) * lv.half_dp64 * c;
    if (sc[5] > sc[4]) {
      const double lo = fmax(lv.p_dyn64, sc[4]), hi = fmin(S.levels[jj + 1].p_dyn64, sc[5]);
      if (hi > lo) dtau += sc[3] * (hi - lo) / (sc[5] - sc[4]);
    }
    return dtau;
  };
  double I[NMU];
  double chi_u, S_u, chi_c = 0.0, S_c = 0.0, chi_d = 0.0, S_d = 0.0;
  level(L, chi_u, S_u);
#pragma unroll
  for (int m = 0; m < NMU; ++m) I[m] = S_u;
  if (L >= 1) level(L - 1, chi_c, S_c);
  for (int j = L - 1; j >= 0; --j) {
    // layer j between level j (S_c, above) and level j+1 (S_u, below)
    const double dtau = layer_dtau(j, chi_c, chi_u);
    double dtau_d = 0.0;
    if (j >= 1) {
      level(j - 1, chi_d, S_d);
      dtau_d = layer_dtau(j - 1, chi_d, chi_c);
    }
#pragma unroll
    for (int m = 0; m < NMU; ++m) {
      if (m < S.n_mu) {
        const double D = dtau / S.mu64[m];
        const double e = exp(-D);
        if (para) {
          // parabolic source through levels j-1, j, j+1 (linear for the top
          // layer): I_j = I_{j+1} e^{-D} + S_j M0 + c1 M1 + c2 M2
          if (!(D > 0.0)) continue;
          double M0, M1, M2;
          exp_moments(D, M0, M1, M2);
          const double du = (S_u - S_c) / D;
          double c1 = du, c2 = 0.0;
          const double Dd = dtau_d / S.mu64[m];
          if (j >= 1 && Dd > 0.0) {
            c2 = (du - (S_c - S_d) / Dd) / (D + Dd);
            c1 = du - c2 * D;
          }
          I[m] = I[m] * e + S_c * M0 + c1 * M1 + c2 * M2;
        } else {
          const double q = (D > 0.0) ? -expm1(-D) / D : 1.0;
          I[m] = I[m] * e + (1.0 - q) * S_c + (q - e) * S_u;
        }
      }
    }
    chi_u = chi_c;
    S_u = S_c;
    chi_c = chi_d;
    S_c = S_d;
  }
  double F = 0.0;
#pragma unroll
  for (int m = 0; m < NMU; ++m)
    if (m < S.n_mu) F += S.wmu64[m] * S.mu64[m] * I[m];
  F *= 2.0 * kPi;
  out[k] = F;
  if (uout) uout[k] = (float)F;
}

cudaError_t launch_forward64(const FwdArgs& a, int max_nmu, int max_nu, cudaStream_t s) {
  if (a.n <= 0) return cudaSuccess;
  dim3 grid((max_nu + kF64Block - 1) / kF64Block, a.n);
  switch (max_nmu) {
    case 1: k_forward64<1><<<grid, kF64Block, 0, s>>>(a); break;
    case 2: k_forward64<2><<<grid, kF64Block, 0, s>>>(a); break;
    case 3: k_forward64<3><<<grid, kF64Block, 0, s>>>(a); break;
    case 4: k_forward64<4><<<grid, kF64Block, 0, s>>>(a); break;
    case 5: k_forward64<5><<<grid, kF64Block, 0, s>>>(a); break;
    case 6: k_forward64<6><<<grid, kF64Block, 0, s>>>(a); break;
    case 7: k_forward64<7><<<grid, kF64Block, 0, s>>>(a); break;
    case 8: k_forward64<8><<<grid, kF64Block, 0, s>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// ------------------------------------------------------------------ bins
// D_m,b = f (R_star/d)^2 sum_m W[b][m] F+_m: the instrument profile and the
// binning as one banded operator (Sects. 2.7-2.8).  One warp per bin row,
// lanes over the row's columns, fixed-order butterfly reduction.
//
// FP32 path: one block per group of up to kBinGroup samples of one setup
// (consecutive in the planner's permutation) and kBinRows rows of W
// (blockIdx.y), so that each row of W is read once for the whole group; each
// sample's sum runs in the same order as it would alone.  (Groups of 2 gave
// the shortest step on the 1024-sample workload: 4 and 8 samples per block
// leave the loads of the rows too serial, 1 reads W once per sample.)  Blocks past the
// groups write NaN rows for samples whose setup index is out of range (they
// are in no group).  FP64 path: one block per sample.
constexpr int kBinGroup = 2;
constexpr int kBinRows = 32;

__global__ void __launch_bounds__(256) k_bins32(FwdArgs a, float* bins, int bins_ld, int group_blocks) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const float qnan = __int_as_float(0x7fc00000);
  int blk = blockIdx.x;
  if (blk >= group_blocks) {
    if (blockIdx.y != 0) return;
    const int i = (blk - group_blocks) * blockDim.x + threadIdx.x;
    if (i < a.n && a.samp[i].setup < 0)
      for (int b = 0; b < bins_ld; ++b) bins[(size_t)i * bins_ld + b] = qnan;
    return;
  }
  const PlanDev* plan = a.plan;
  int g = -1, s0 = 0, ns = 0;
  for (int q = 0; q < plan->n_setups; ++q) {
    const int c = plan->count[q], nb = (c + kBinGroup - 1) / kBinGroup;
    if (blk < nb) {
      g = q;
      s0 = plan->first[q] + blk * kBinGroup;
      ns = min(kBinGroup, c - blk * kBinGroup);
      break;
    }
    blk -= nb;
  }
  if (g < 0) return;   // beyond the groups of this batch
  const SetupDev& S = *a.setups[g];
  const float* F[kBinGroup];
  float* out[kBinGroup];
  float scale_hi[kBinGroup], scale_lo[kBinGroup];
  bool bad[kBinGroup];
#pragma unroll
  for (int k = 0; k < kBinGroup; ++k) {
    const int i = a.perm[s0 + min(k, ns - 1)];
    F[k] = a.highres + (size_t)i * a.highres_ld;
    out[k] = bins + (size_t)i * bins_ld;
    scale_hi[k] = a.samp[i].scale32[0];
    scale_lo[k] = a.samp[i].scale32[1];
    bad[k] = a.samp[i].status != 0;
  }
  const int b_end = min(S.n_bins, (int)(blockIdx.y + 1) * kBinRows);
  for (int b = blockIdx.y * kBinRows + warp; b < b_end; b += nw) {
    const long long r0 = S.w_rowptr[b], r1 = S.w_rowptr[b + 1];
    const int c0 = S.w_col0[b];
    if constexpr (HR2_BOUNDS_CHECK) {
      // the row's weights and the F+ points it reads
      if (!bounds_ok(r0 >= 0 && r1 >= r0 && r1 <= S.w_nnz && c0 >= 0 && c0 + (r1 - r0) <= S.n_nu &&
                         S.n_nu <= a.highres_ld && b < bins_ld,
                     lane == 0 ? a.err : nullptr))
        continue;
    }
    float acc[kBinGroup];
#pragma unroll
    for (int k = 0; k < kBinGroup; ++k) acc[k] = 0.f;
#pragma unroll 2
    for (long long t = r0 + lane; t < r1; t += 32) {
      const float w = S.w32[t];
      const long long c = c0 + (t - r0);
#pragma unroll
      for (int k = 0; k < kBinGroup; ++k)
        if (k < ns) acc[k] = fmaf(w, F[k][c], acc[k]);
    }
#pragma unroll
    for (int k = 0; k < kBinGroup; ++k) {
      if (k >= ns) break;
      float v = acc[k];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      // v f (R/d)^2 with the scale as an FP32 head and tail (FP64 arithmetic
      // here would run on the SM's few FP64 units once per row)
      if (lane == 0) out[k][b] = bad[k] ? qnan : fmaf(v, scale_hi[k], v * scale_lo[k]);
    }
  }
}

__global__ void __launch_bounds__(256) k_bins64(FwdArgs a, float* bins, int bins_ld) {
  const int i = blockIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const SampleDev& sd = a.samp[i];
  float* out = bins + (size_t)i * bins_ld;
  const float qnan = __int_as_float(0x7fc00000);
  if (sd.setup < 0) {
    for (int b = threadIdx.x; b < bins_ld; b += blockDim.x) out[b] = qnan;
    return;
  }
  const SetupDev& S = *a.setups[sd.setup];
  if (sd.status != 0) {
    for (int b = threadIdx.x; b < S.n_bins; b += blockDim.x) out[b] = qnan;
    return;
  }
  for (int b = warp; b < S.n_bins; b += nw) {
    const long long r0 = S.w_rowptr[b], r1 = S.w_rowptr[b + 1];
    const int c0 = S.w_col0[b];
    const double* F = a.highres64 + (size_t)i * a.highres64_ld + c0;
    double acc = 0.0;
    for (long long t = r0 + lane; t < r1; t += 32) acc += S.w64[t] * F[t - r0];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) out[b] = (float)(acc * sd.scale);
  }
}

cudaError_t launch_bins(const FwdArgs& a, float* bins, int bins_ld, bool fp64, cudaStream_t s) {
  if (a.n <= 0) return cudaSuccess;
  if (fp64) {
    k_bins64<<<a.n, 256, 0, s>>>(a, bins, bins_ld);
  } else {
    // groups: at most n / kBinGroup + one partial group per setup
    const int group_blocks = (a.n + kBinGroup - 1) / kBinGroup + a.n_setups;
    const dim3 grid(group_blocks + (a.n + 255) / 256, (bins_ld + kBinRows - 1) / kBinRows);
    k_bins32<<<grid, 256, 0, s>>>(a, bins, bins_ld, group_blocks);
  }
  return cudaGetLastError();
}

// ------------------------------------------------------------------ lnL
// ln L = sum_j -(D_j - D_m,j)^2 / (2 s_j^2) - ln(2 pi s_j^2) / 2, with
// s_j^2 = sigma_j^2 (+ 10^eps) (Eqs. 19, 22-23).  One warp per sample, FP64,
// fixed-order butterfly reduction.  Without error inflation (no eps, or a
// non-finite one) the normalisation sum and 1 / (2 sigma_j^2) come from the
// observation's precomputed terms, so a bin costs one subtraction and one FMA.
__global__ void __launch_bounds__(256) k_lnl(LnlArgs a) {
  const int lane = threadIdx.x & 31;
  const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (i >= a.n) return;
  const int g = a.setup_of_sample[i];
  if (g < 0 || g >= a.n_setups) {
    if (lane == 0) a.lnl[i] = -HUGE_VAL;
    return;
  }
  const SetupDev& S = *a.setups[g];
  const double eps = a.log_eps ? a.log_eps[i] : __longlong_as_double(0x7ff8000000000000ll);
  const float* m = a.bins + (size_t)i * a.bins_ld;
  double acc = 0.0;
  int bad = 0;
  if (!isfinite(eps)) {
    for (int b = lane; b < S.n_bins; b += 32) {
      const double dm = (double)m[b];
      if (!isfinite(dm)) bad = 1;
      const double r = S.obs_D[b] - dm;
      acc = fma(-r * r, S.obs_inv2s2[b], acc);
    }
  } else {
    const double add = exp10(eps);
    for (int b = lane; b < S.n_bins; b += 32) {
      const double dm = (double)m[b];
      if (!isfinite(dm)) bad = 1;
      const double sg = S.obs_sigma[b];
      const double s2 = sg * sg + add;
      const double r = S.obs_D[b] - dm;
      acc += -r * r / (2.0 * s2) - 0.5 * log(2.0 * kPi * s2);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  bad = __reduce_or_sync(0xffffffffu, bad);
  if (!isfinite(eps)) acc += *S.obs_lnorm;
  if (lane == 0) a.lnl[i] = bad ? -HUGE_VAL : acc;
}

// The observation's model-independent likelihood terms: 1 / (2 sigma_b^2)
// and sum_b -ln(2 pi sigma_b^2) / 2 (one warp, FP64, fixed order).
__global__ void k_obs_terms(const double* sigma, int n_bins, double* inv2s2, double* lnorm) {
  const int lane = threadIdx.x;
  double acc = 0.0;
  for (int b = lane; b < n_bins; b += 32) {
    const double s2 = sigma[b] * sigma[b];
    inv2s2[b] = 1.0 / (2.0 * s2);
    acc += -0.5 * log(2.0 * kPi * s2);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) *lnorm = acc;
}

cudaError_t launch_obs_terms(const double* sigma, int n_bins, double* inv2s2, double* lnorm, cudaStream_t s) {
  k_obs_terms<<<1, 32, 0, s>>>(sigma, n_bins, inv2s2, lnorm);
  return cudaGetLastError();
}

cudaError_t launch_lnl(const LnlArgs& a, cudaStream_t s) {
  if (a.n <= 0) return cudaSuccess;
  k_lnl<<<(a.n + 7) / 8, 256, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace hr2
