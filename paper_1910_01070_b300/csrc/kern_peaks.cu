// kern_peaks.cu -- microbenchmarks of the arithmetic units the forward
// kernel's roofline is taken against: the special-function unit (ex2 and rcp,
// approximate, flush-to-zero: the forms k_forward32 issues) and the FP32 FMA
// pipe (scalar and packed f32x2).  Each kernel runs many independent
// dependency chains per thread at full occupancy, so that the unit, not
// latency, bounds it; one thread per CTA records its SM and clock64 at both
// ends, which gives each SM's busy span in its own cycles.
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "hr2_internal.cuh"

namespace hr2 {
namespace {

constexpr int kChains = 16;          // independent chains per thread
constexpr int kPeakThreads = 256;    // per CTA
constexpr int kPeakCtasPerSm = 8;    // 2048 threads per SM

__device__ __forceinline__ float pk_ex2(float x) {
  float y;
  asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float pk_rcp(float x) {
  float y;
  asm volatile("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ unsigned long long pk_fma2(unsigned long long a, unsigned long long b,
                                                      unsigned long long c) {
  unsigned long long d;
  asm volatile("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
// Per CTA: {clock64 at the start, clock64 at the end, SM index}.
__device__ __forceinline__ void stamp(long long* st, bool end) {
  if (threadIdx.x == 0) {
    st[3 * blockIdx.x + (end ? 1 : 0)] = clock64();
    if (end) {
      unsigned smid;
      asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
      st[3 * blockIdx.x + 2] = smid;
    }
  }
}

// kind 0: half the chains y <- 2^(-y), half y <- 1/y + 1 (the forward
//         kernel's mix of the two special functions; ops counts both),
//         kind 1: y <- 1/y + 1 (rcp; fixed point the golden ratio),
//         kind 2: y <- 2^(-y) (ex2; fixed point 0.641), kind 3: y <- y a + b
//         scalar FFMA, kind 4: the same as packed f32x2 FMA.  Each special-
//         function step carries one FP32 addition, so the chains cannot be
//         shortened algebraically and the unit, not issue, bounds them.
template <int KIND>
__global__ void __launch_bounds__(kPeakThreads) k_unit_rate(long long iters, float* out, long long* st) {
  float y[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) y[c] = 1.25f + 1e-6f * (float)(threadIdx.x + c);
  __syncthreads();
  stamp(st, false);
  for (long long it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
      if constexpr (KIND == 0) y[c] = (c & 1) ? pk_rcp(y[c]) + 1.f : pk_ex2(0.f - y[c]);
      else if constexpr (KIND == 1) y[c] = pk_rcp(y[c]) + 1.f;
      else if constexpr (KIND == 2) y[c] = pk_ex2(0.f - y[c]);
      else if constexpr (KIND == 3) y[c] = fmaf(y[c], 0.5f, 0.25f);
    }
    if constexpr (KIND == 4) {
#pragma unroll
      for (int c = 0; c < kChains; c += 2) {
        unsigned long long v;
        asm("mov.b64 %0, {%1, %2};" : "=l"(v) : "f"(y[c]), "f"(y[c + 1]));
        const unsigned long long a = 0x3f0000003f000000ull, b = 0x3e8000003e800000ull;   // {0.5, 0.5}, {0.25, 0.25}
        v = pk_fma2(v, a, b);
        asm("mov.b64 {%0, %1}, %2;" : "=f"(y[c]), "=f"(y[c + 1]) : "l"(v));
      }
    }
  }
  __syncthreads();
  stamp(st, true);
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += y[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace
}  // namespace hr2

using namespace hr2;

extern "C" int hr2_measure_unit_rate(int device, int kind, long long iters, hr2_unit_rate* out) {
  if (!out || kind < 0 || kind >= HR2_UNIT_KINDS || iters < 1) return HR2_EINVAL;
  if (cudaSetDevice(device) != cudaSuccess) return HR2_ECUDA;
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return HR2_ECUDA;
  const int n_sm = prop.multiProcessorCount;
  const int grid = n_sm * kPeakCtasPerSm;
  float* d_out = nullptr;
  long long* d_st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = HR2_OK;
  if (cudaMalloc(&d_out, sizeof(float) * (size_t)grid * kPeakThreads) != cudaSuccess ||
      cudaMalloc(&d_st, sizeof(long long) * 3 * (size_t)grid) != cudaSuccess ||
      cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    rc = HR2_ECUDA;
  }
  auto launch = [&](long long it) {
    switch (kind) {
      case HR2_UNIT_EX2_RCP: k_unit_rate<0><<<grid, kPeakThreads>>>(it, d_out, d_st); break;
      case HR2_UNIT_RCP: k_unit_rate<1><<<grid, kPeakThreads>>>(it, d_out, d_st); break;
      case HR2_UNIT_EX2: k_unit_rate<2><<<grid, kPeakThreads>>>(it, d_out, d_st); break;
      case HR2_UNIT_FFMA: k_unit_rate<3><<<grid, kPeakThreads>>>(it, d_out, d_st); break;
      default: k_unit_rate<4><<<grid, kPeakThreads>>>(it, d_out, d_st); break;
    }
  };
  float ms = 0.f;
  if (rc == HR2_OK) {
    launch(std::max(1ll, iters / 16));   // warm-up
    cudaEventRecord(e0);
    launch(iters);
    cudaEventRecord(e1);
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) rc = HR2_ECUDA;
  }
  if (rc == HR2_OK) {
    std::vector<long long> st(3 * (size_t)grid);
    if (cudaMemcpy(st.data(), d_st, sizeof(long long) * st.size(), cudaMemcpyDeviceToHost) != cudaSuccess) {
      rc = HR2_ECUDA;
    } else {
      // SM cycles of the run: per SM, its first CTA's start to its last CTA's
      // end (clock64 counts per SM), the median over SMs
      // (SM indices may be sparse: %smid runs up to %nsmid, which can exceed the SM count)
      long long n_id = 0;
      for (int b = 0; b < grid; ++b) n_id = std::max(n_id, st[3 * b + 2] + 1);
      std::vector<long long> lo((size_t)n_id, -1), hi((size_t)n_id, -1);
      for (int b = 0; b < grid; ++b) {
        const long long sm = st[3 * b + 2];
        if (sm < 0 || sm >= n_id) continue;
        if (lo[sm] < 0 || st[3 * b] < lo[sm]) lo[sm] = st[3 * b];
        if (hi[sm] < 0 || st[3 * b + 1] > hi[sm]) hi[sm] = st[3 * b + 1];
      }
      std::vector<double> cyc;
      for (long long m = 0; m < n_id; ++m)
        if (lo[m] >= 0 && hi[m] > lo[m]) cyc.push_back((double)(hi[m] - lo[m]));
      std::sort(cyc.begin(), cyc.end());
      const double cycles = cyc.empty() ? 0.0 : cyc[cyc.size() / 2];
      // every chain step is one operation of the measured kind (one packed
      // instruction per two chains for HR2_UNIT_FFMA2, counted as two FMAs)
      const double ops = (double)grid * kPeakThreads * (double)iters * kChains;
      out->ms = ms;
      out->ops = ops;
      out->ops_per_s = ops / (ms * 1e-3);
      out->sm_ghz = cycles / (ms * 1e6);
      out->ops_per_clk_sm = cycles > 0 ? ops / n_sm / cycles : 0.0;
      out->n_sm = n_sm;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(d_out);
  cudaFree(d_st);
  return rc;
}
