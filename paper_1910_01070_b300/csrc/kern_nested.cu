// kern_nested.cu -- evidence bookkeeping of nested sampling on the device
// (Sect. 3.2, after Skilling 2004): absorb scored candidates into the live
// set, accumulate ln Z and the information H in FP64, add the live remainder.
//
// The live set stays on the device, so a sampler's loop
//   propose -> forward_model_batch -> log_likelihood_batch -> absorb
// needs no host round trip per replacement.  One CTA processes the
// candidates in order; every replacement is followed by a block-wide argmin
// over the live likelihoods.  All threads carry the same running sums (the
// values they reduce and compare are the same), so the control flow is
// uniform.
#include <math.h>

#include "hr2_internal.cuh"

namespace hr2 {

constexpr int kNsThreads = 512;

// ln(e^a + e^b); -inf is the empty sum
__device__ __forceinline__ double log_add(double a, double b) {
  if (a == -INFINITY) return b;
  if (b == -INFINITY) return a;
  const double m = fmax(a, b);
  return m + log(exp(a - m) + exp(b - m));
}

// Fold a point of likelihood e^lnl and prior weight e^log_w into ln Z and H.
// H = sum_k p_k ln L_k - ln Z (p_k = L_k w_k / Z), updated in Skilling's
// running form: H' = e^(lw - Z') lnl + e^(Z - Z') (H + Z) - Z'.
__device__ __forceinline__ void ns_add(double& log_z, double& info, double lnl, double log_w) {
  const double lw = lnl + log_w;
  const double z_new = log_add(log_z, lw);
  double h = 0.0;
  if (lw > -INFINITY) h += exp(lw - z_new) * lnl;
  if (log_z > -INFINITY) h += exp(log_z - z_new) * (info + log_z);
  info = h - z_new;
  log_z = z_new;
}

// Smallest live value and its index (ties: lowest index; NaN counts as
// +inf), broadcast to every thread of the block.
__device__ void block_argmin(const double* v, int n, double& best_v, int& best_i) {
  __shared__ double s_v[kNsThreads / 32];
  __shared__ int s_i[kNsThreads / 32];
  double bv = INFINITY;
  int bi = 0x7fffffff;
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    const double x = isnan(v[j]) ? INFINITY : v[j];
    if (x < bv || (x == bv && j < bi)) {
      bv = x;
      bi = j;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
    const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
    if (ov < bv || (ov == bv && oi < bi)) {
      bv = ov;
      bi = oi;
    }
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  __syncthreads();   // earlier readers of s_v / s_i are done
  if (lane == 0) {
    s_v[warp] = bv;
    s_i[warp] = bi;
  }
  __syncthreads();
  bv = lane < nw ? s_v[lane] : INFINITY;
  bi = lane < nw ? s_i[lane] : 0x7fffffff;
  for (int o = 16; o > 0; o >>= 1) {
    const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
    const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
    if (ov < bv || (ov == bv && oi < bi)) {
      bv = ov;
      bi = oi;
    }
  }
  best_v = bv;
  best_i = bi;
}

// Largest live value (NaN ignored), broadcast to every thread.
__device__ double block_max(const double* v, int n) {
  __shared__ double s_m[kNsThreads / 32];
  double m = -INFINITY;
  for (int j = threadIdx.x; j < n; j += blockDim.x) m = fmax(m, v[j]);
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0) s_m[warp] = m;
  __syncthreads();
  m = lane < nw ? s_m[lane] : -INFINITY;
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

__global__ void __launch_bounds__(kNsThreads) k_ns_absorb(int n_live, double* live_lnl, double* live_theta,
                                                          int n_cand, const double* cand_lnl,
                                                          const double* cand_theta, hr2_ns_state* st,
                                                          double* dead_lnl, double* dead_logw, double* dead_theta,
                                                          long long dead_cap) {
  long long n_dead = st->n_dead, n_seen = st->n_seen;
  double log_z = st->log_z, info = st->info;
  const double lw1 = log(-expm1(-1.0 / (double)n_live));   // ln(1 - e^(-1/N))
  double wv;
  int worst;
  block_argmin(live_lnl, n_live, wv, worst);
  for (int c = 0; c < n_cand; ++c) {
    if (n_dead >= dead_cap) break;
    ++n_seen;
    const double cl = cand_lnl[c];
    if (!(cl > wv)) continue;
    const long long i = n_dead + 1;
    const double log_w = -(double)(i - 1) / (double)n_live + lw1;
    for (int t = threadIdx.x; t < HR2_NPARAM; t += blockDim.x) {
      dead_theta[n_dead * HR2_NPARAM + t] = live_theta[(size_t)worst * HR2_NPARAM + t];
      live_theta[(size_t)worst * HR2_NPARAM + t] = cand_theta[(size_t)c * HR2_NPARAM + t];
    }
    if (threadIdx.x == 0) {
      dead_lnl[n_dead] = wv;
      dead_logw[n_dead] = log_w;
      live_lnl[worst] = cl;
    }
    ns_add(log_z, info, wv, log_w);
    n_dead = i;
    __syncthreads();   // the replaced live value is visible to the next argmin
    block_argmin(live_lnl, n_live, wv, worst);
  }
  const double vmax = block_max(live_lnl, n_live);
  if (threadIdx.x == 0) {
    st->n_dead = n_dead;
    st->n_seen = n_seen;
    st->log_z = log_z;
    st->info = info;
    st->log_x = -(double)n_dead / (double)n_live;
    st->lnl_min = wv;
    st->lnl_max = vmax;
  }
}

// Live remainder: each live point with weight X_n / N, in index order.
__global__ void k_ns_finalize(int n_live, const double* live_lnl, const hr2_ns_state* st, double* out) {
  double log_z = st->log_z, info = st->info;
  const double log_w = -(double)st->n_dead / (double)n_live - log((double)n_live);
  for (int j = 0; j < n_live; ++j) ns_add(log_z, info, live_lnl[j], log_w);
  out[0] = log_z;
  out[1] = info;
}

cudaError_t launch_ns_init(hr2_ns_state* st, cudaStream_t s) {
  k_ns_init<<<1, 1, 0, s>>>(st);
  return cudaGetLastError();
}

cudaError_t launch_ns_absorb(int n_live, double* live_lnl, double* live_theta, int n_cand, const double* cand_lnl,
                             const double* cand_theta, hr2_ns_state* st, double* dead_lnl, double* dead_logw,
                             double* dead_theta, long long dead_cap, cudaStream_t s) {
  k_ns_absorb<<<1, kNsThreads, 0, s>>>(n_live, live_lnl, live_theta, n_cand, cand_lnl, cand_theta, st, dead_lnl,
                                       dead_logw, dead_theta, dead_cap);
  return cudaGetLastError();
}

cudaError_t launch_ns_finalize(int n_live, const double* live_lnl, const hr2_ns_state* st, double* out,
                               cudaStream_t s) {
  k_ns_finalize<<<1, 1, 0, s>>>(n_live, live_lnl, st, out);
  return cudaGetLastError();
}

}  // namespace hr2
