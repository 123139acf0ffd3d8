// kern_nested.cu -- evidence bookkeeping of nested sampling on the device
// (Sect. 3.2, after Skilling 2004): absorb scored candidates into the live
// set, accumulate ln Z and the information H in FP64, add the live remainder.
//
// The live set stays on the device, so a sampler's loop
//   propose -> forward_model_batch -> log_likelihood_batch -> absorb
// needs no host round trip per replacement.  The candidates are consumed
// strictly in order, so the absorb step is one warp: integer keys of the
// live likelihoods sit in shared memory (when they fit), the candidates'
// likelihoods are fetched 32 at a time and handed along by shuffles, and
// after every replacement the warp takes the argmin over the keys.  ln Z and
// H (FP64, of which the SM has few units) take the call's dead points in one
// fixed-order warp reduction once the replacements are known.  All lanes
// carry the same values, so the control flow is uniform.
#include <math.h>

#include "hr2_internal.cuh"

namespace hr2 {

// live likelihoods held in shared memory by the absorb warp, up to this many
constexpr int kNsLiveSmem = 4096;
static_assert(HR2_NPARAM <= 64, "the absorb warp moves a parameter row as two elements per lane");

// Fold points k = 0 .. n-1 of likelihood e^lnl[k] and prior weight
// e^(logw ? logw[k] : logw_c) into ln Z and H, on every lane of the warp.
// Z' = Z + sum_k L_k w_k and H' = sum over all points of p ln L - ln Z'
// (p = L w / Z'), the closed form of Skilling's one-point-at-a-time update
//   Z' = ln(e^Z + L w),  H' = e^(lw - Z') lnl + e^(Z - Z') (H + Z) - Z',
// evaluated as a fixed-order warp reduction instead of a chain of FP64
// exponentials and logarithms (~3.6 us per point on this SM); the two agree
// to rounding.  A term with lnL = -inf adds nothing; a NaN likelihood
// makes ln Z NaN, as in the one-point form.
__device__ void ns_fold(double& log_z, double& info, long long n, const double* lnl, const double* logw,
                        double logw_c) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const double z0 = log_z, h0 = info;
  double m = -INFINITY;
  for (long long k = lane; k < n; k += 32) m = fmax(m, lnl[k] + (logw ? logw[k] : logw_c));
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(full, m, o));
  m = fmax(m, z0);
  double sum = 0.0;
  for (long long k = lane; k < n; k += 32) {
    const double lw = lnl[k] + (logw ? logw[k] : logw_c);
    if (lw != -INFINITY) sum += exp(lw - m);
  }
  for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(full, sum, o);
  if (z0 != -INFINITY) sum += exp(z0 - m);
  const double z1 = m + log(sum);   // -inf when every term is empty
  double t = 0.0;
  for (long long k = lane; k < n; k += 32) {
    const double l = lnl[k], lw = l + (logw ? logw[k] : logw_c);
    if (lw > -INFINITY) t += exp(lw - z1) * l;
  }
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(full, t, o);
  if (z0 > -INFINITY) t += exp(z0 - z1) * (h0 + z0);
  info = t - z1;
  log_z = z1;
}

// Order-preserving integer key of a live likelihood, so that the warp's
// argmin and the candidates' test run on integer compares (the SM's FP64
// units are few): NaN counts as +inf, -0 as +0.
constexpr long long kNsKeyInf = 0x7ff0000000000000LL;
__device__ __forceinline__ long long ns_key(double x) {
  const long long b = __double_as_longlong(x);
  const long long mag = b & 0x7fffffffffffffffLL;
  if (mag > kNsKeyInf) return kNsKeyInf;
  if (mag == 0) return 0;
  return b < 0 ? (b ^ 0x7fffffffffffffffLL) : b;
}
__device__ __forceinline__ double ns_unkey(long long k) {
  return __longlong_as_double(k < 0 ? (k ^ 0x7fffffffffffffffLL) : k);
}
// a candidate's key: a NaN candidate is never above the live minimum
__device__ __forceinline__ long long ns_cand_key(double x) {
  return isnan(x) ? (long long)0x8000000000000000ULL : ns_key(x);
}

// Key of the smallest live value and its index (ties: lowest index), on
// every lane; keys from shared memory, or formed from the values in place.
template <bool SMEM>
__device__ __forceinline__ void warp_argmin(const long long* key, const double* v, int n, long long& best_k,
                                            int& best_i) {
  const int lane = threadIdx.x & 31;
  long long bk = 0x7fffffffffffffffLL;
  int bi = 0x7fffffff;
  for (int j = lane; j < n; j += 32) {
    const long long k = SMEM ? key[j] : ns_key(v[j]);
    if (k < bk) {   // a lane visits its indices in increasing order
      bk = k;
      bi = j;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    const long long ok = __shfl_xor_sync(0xffffffffu, bk, o);
    const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
    if (ok < bk || (ok == bk && oi < bi)) {
      bk = ok;
      bi = oi;
    }
  }
  best_k = bk;
  best_i = bi;
}

// Largest live value (NaN ignored), on every lane.
__device__ __forceinline__ double warp_max(const double* v, int n) {
  double m = -INFINITY;
  for (int j = threadIdx.x & 31; j < n; j += 32) m = fmax(m, v[j]);
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  return m;
}

__global__ void k_ns_init(hr2_ns_state* st) {
  hr2_ns_state s{};
  s.n_dead = 0;
  s.n_seen = 0;
  s.log_z = -INFINITY;
  s.info = 0.0;
  s.log_x = 0.0;
  s.lnl_min = INFINITY;
  s.lnl_max = -INFINITY;
  *st = s;
}

template <bool SMEM>
__global__ void __launch_bounds__(32) k_ns_absorb(int n_live, double* live_lnl, double* live_theta, int n_cand,
                                                  const double* cand_lnl, const double* cand_theta,
                                                  hr2_ns_state* st, double* dead_lnl, double* dead_logw,
                                                  double* dead_theta, long long dead_cap) {
  __shared__ long long s_key[SMEM ? kNsLiveSmem : 1];
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  if (SMEM)
    for (int j = lane; j < n_live; j += 32) s_key[j] = ns_key(live_lnl[j]);
  __syncwarp();
  const long long dead0 = st->n_dead;
  long long n_dead = dead0, n_seen = st->n_seen;
  const double lw1 = log(-expm1(-1.0 / (double)n_live));   // ln(1 - e^(-1/N))
  long long wk;
  int worst;
  warp_argmin<SMEM>(s_key, live_lnl, n_live, wk, worst);
  bool full_cap = false;
  for (int c0 = 0; c0 < n_cand && !full_cap; c0 += 32) {
    const double mine = c0 + lane < n_cand ? cand_lnl[c0 + lane] : 0.0;
    const long long mine_k = ns_cand_key(mine);
    const int m = min(32, n_cand - c0);
    for (int k = 0; k < m; ++k) {
      if (n_dead >= dead_cap) {
        full_cap = true;
        break;
      }
      ++n_seen;
      if (!(__shfl_sync(full, mine_k, k) > wk)) continue;   // not strictly above the live minimum
      const double cl = __shfl_sync(full, mine, k);
      const long long c = c0 + k;
      // the leaving point's parameters go to the dead list and the
      // candidate's take its place (HR2_NPARAM <= 64: two elements per
      // lane); loaded here, stored after the next argmin, which does not
      // need them (a lane stores and later loads only its own elements)
      const size_t lrow = (size_t)worst * HR2_NPARAM, crow = (size_t)c * HR2_NPARAM,
                   drow = (size_t)n_dead * HR2_NPARAM;
      const bool two = lane + 32 < HR2_NPARAM;
      const double a0 = live_theta[lrow + lane], b0 = cand_theta[crow + lane];
      const double a1 = two ? live_theta[lrow + lane + 32] : 0.0, b1 = two ? cand_theta[crow + lane + 32] : 0.0;
      if (lane == 0) {
        // dead point i = n_dead + 1: its likelihood; ln w_i, ln Z and H
        // follow after the loop, in the same order
        dead_lnl[n_dead] = ns_unkey(wk);
        live_lnl[worst] = cl;
        if (SMEM) s_key[worst] = ns_key(cl);
      }
      ++n_dead;
      __syncwarp();   // the replaced live value is visible to the next argmin
      warp_argmin<SMEM>(s_key, live_lnl, n_live, wk, worst);
      dead_theta[drow + lane] = a0;
      live_theta[lrow + lane] = b0;
      if (two) {
        dead_theta[drow + lane + 32] = a1;
        live_theta[lrow + lane + 32] = b1;
      }
    }
  }
  // ln w_i = -(i-1)/N + ln(1 - e^(-1/N)) of the call's dead points, one per lane
  for (long long d = dead0 + lane; d < n_dead; d += 32) dead_logw[d] = -(double)d / (double)n_live + lw1;
  __syncwarp();   // the dead-list entries are visible to every lane
  double log_z = st->log_z, info = st->info;
  if (n_dead > dead0) ns_fold(log_z, info, n_dead - dead0, dead_lnl + dead0, dead_logw + dead0, 0.0);
  const double vmax = warp_max(live_lnl, n_live);
  if (lane == 0) {
    st->n_dead = n_dead;
    st->n_seen = n_seen;
    st->log_z = log_z;
    st->info = info;
    st->log_x = -(double)n_dead / (double)n_live;
    st->lnl_min = ns_unkey(wk);
    st->lnl_max = vmax;
  }
}

// Live remainder: each live point with weight X_n / N.
__global__ void __launch_bounds__(32) k_ns_finalize(int n_live, const double* live_lnl, const hr2_ns_state* st,
                                                    double* out) {
  double log_z = st->log_z, info = st->info;
  const double log_w = -(double)st->n_dead / (double)n_live - log((double)n_live);
  ns_fold(log_z, info, n_live, live_lnl, nullptr, log_w);
  if ((threadIdx.x & 31) == 0) {
    out[0] = log_z;
    out[1] = info;
  }
}

// ------------------------------------------------------------ proposals
// Candidates of the minimal sampler: uniform in the bounding box of the live
// points, widened by `enlarge` x its span on each side and clipped to the
// prior box; a parameter with lo == hi stays at lo.  The uniform deviates come
// from SplitMix64 (Steele, Lea & Flood 2014, the finaliser of a Weyl sequence)
// at counter values counter + i HR2_NPARAM + p, top 53 bits -> [0, 1).
__device__ __forceinline__ double ns_uniform(unsigned long long seed, unsigned long long ctr) {
  unsigned long long z = seed + (ctr + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return (double)(z >> 11) * 0x1.0p-53;
}

// block p: the live points' range of parameter p -> the proposal box
__global__ void __launch_bounds__(256) k_ns_box(int n_live, const double* live_theta, const double* lo,
                                                const double* hi, double enlarge, double* box) {
  __shared__ double s_mn[8], s_mx[8];
  const int p = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double mn = INFINITY, mx = -INFINITY;
  for (int j = threadIdx.x; j < n_live; j += blockDim.x) {
    const double v = live_theta[(size_t)j * HR2_NPARAM + p];
    mn = fmin(mn, v);
    mx = fmax(mx, v);
  }
  for (int o = 16; o > 0; o >>= 1) {
    mn = fmin(mn, __shfl_xor_sync(0xffffffffu, mn, o));
    mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  }
  if (lane == 0) {
    s_mn[warp] = mn;
    s_mx[warp] = mx;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
      mn = fmin(mn, s_mn[w]);
      mx = fmax(mx, s_mx[w]);
    }
    const double span = mx - mn;
    box[2 * p] = fmax(lo[p], mn - enlarge * span);
    box[2 * p + 1] = fmin(hi[p], mx + enlarge * span);
  }
}

__global__ void __launch_bounds__(256) k_ns_draw(int n, const double* lo, const double* hi, const double* box,
                                                 unsigned long long seed, unsigned long long counter, double* out) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)n * HR2_NPARAM) return;
  const int p = (int)(idx % HR2_NPARAM);
  double v = lo[p];
  if (hi[p] > lo[p]) {
    const double a = box[2 * p], b = box[2 * p + 1];
    v = a + (b - a) * ns_uniform(seed, counter + (unsigned long long)idx);
  }
  out[idx] = v;
}

cudaError_t launch_ns_propose(int n_live, const double* live_theta, const double* lo, const double* hi,
                              double enlarge, int n, double* box, double* out, unsigned long long seed,
                              unsigned long long counter, cudaStream_t s) {
  k_ns_box<<<HR2_NPARAM, 256, 0, s>>>(n_live, live_theta, lo, hi, enlarge, box);
  if (n > 0) {
    const long long total = (long long)n * HR2_NPARAM;
    k_ns_draw<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(n, lo, hi, box, seed, counter, out);
  }
  return cudaGetLastError();
}

cudaError_t launch_ns_init(hr2_ns_state* st, cudaStream_t s) {
  k_ns_init<<<1, 1, 0, s>>>(st);
  return cudaGetLastError();
}

cudaError_t launch_ns_absorb(int n_live, double* live_lnl, double* live_theta, int n_cand, const double* cand_lnl,
                             const double* cand_theta, hr2_ns_state* st, double* dead_lnl, double* dead_logw,
                             double* dead_theta, long long dead_cap, cudaStream_t s) {
  if (n_live <= kNsLiveSmem)
    k_ns_absorb<true><<<1, 32, 0, s>>>(n_live, live_lnl, live_theta, n_cand, cand_lnl, cand_theta, st, dead_lnl,
                                       dead_logw, dead_theta, dead_cap);
  else
    k_ns_absorb<false><<<1, 32, 0, s>>>(n_live, live_lnl, live_theta, n_cand, cand_lnl, cand_theta, st, dead_lnl,
                                        dead_logw, dead_theta, dead_cap);
  return cudaGetLastError();
}

cudaError_t launch_ns_finalize(int n_live, const double* live_lnl, const hr2_ns_state* st, double* out,
                               cudaStream_t s) {
  k_ns_finalize<<<1, 32, 0, s>>>(n_live, live_lnl, st, out);
  return cudaGetLastError();
}

}  // namespace hr2
