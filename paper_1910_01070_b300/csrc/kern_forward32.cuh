// kern_forward32.cuh -- the FP32 forward kernel k_forward32 (level sweep of
// one sample on one wavenumber tile per warp) and its launch templates,
// instantiated per angle-node count in kern_fwd32_inst.cu so that the
// instantiations compile in parallel.
#pragma once
#include <math.h>
#include <stddef.h>

#include "hr2_internal.cuh"

namespace hr2 {


__device__ __forceinline__ float ex2f(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rcpf(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// ---------------------------------------------------------- FP32 forward
// Packed two-wide FP32 arithmetic (Blackwell f32x2): each lane carries two
// neighbouring wavenumbers through the whole level sweep, so every FMA, add
// and multiply of the path issues once for both.
typedef unsigned long long v2;
__device__ __forceinline__ v2 pk(float a, float b) {
  v2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ v2 pk(float a) { return pk(a, a); }
__device__ __forceinline__ float2 up(v2 r) {
  float2 a;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a.x), "=f"(a.y) : "l"(r));
  return a;
}
__device__ __forceinline__ v2 fma2(v2 a, v2 b, v2 c) {
  v2 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ v2 add2(v2 a, v2 b) {
  v2 d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ v2 sub2(v2 a, v2 b) {
  v2 d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ v2 mul2(v2 a, v2 b) {
  v2 d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ v2 ex2_2(v2 x) {
  const float2 f = up(x);
  return pk(ex2f(f.x), ex2f(f.y));
}
__device__ __forceinline__ v2 rcp_2(v2 x) {
  const float2 f = up(x);
  return pk(rcpf(f.x), rcpf(f.y));
}
__device__ __forceinline__ v2 h2f2(unsigned int h) {
  const float2 f = __half22float2(*reinterpret_cast<const __half2*>(&h));
  return pk(f.x, f.y);
}
__device__ __forceinline__ unsigned int ldh2(const __half* p) {
  return __ldg(reinterpret_cast<const unsigned int*>(p));
}

// log2(10) as an FP32 head and tail
constexpr float kL2Hi = 3.32192802f;
constexpr float kL2Lo = (float)(kLog2_10 - (double)kL2Hi);
// below this optical thickness D the parabolic-source moments come from
// their power series instead of from differences of exponentials
constexpr float kThinD = 0.25f;
// below this D the linear-source layer factor 1 - e^{-D} comes from its
// series D - D^2/2 + D^3/6 (truncation <= D^3/24 = 1.3e-6 relative); above it
// from the difference of the two exponentials (rounding ~2^-22 / D <= 7.6e-6
// relative, ~1e-6 typical)
constexpr float kThinLin = 0.03125f;
constexpr float kLog2eF = 1.44269504088896341f;

// One warp computes one sample on one kTileNu-point wavenumber tile (kPairs
// packed pairs of points per lane), sweeping the levels from the top (j = 0)
// to the bottom (j = L):
//   log10 sigma_s: bilinear in (T, log10 p) written as corner 00 plus
//                  weighted differences (exact partition of unity)
//   chi_j = sum_s x_s c sigma_s + CIA     (Sects. 2.3, 2.8; 2^(A_s + ...))
//   dtau_l = (chi_l + chi_{l+1}) (p_{l+1} - p_l) / 2
//   S_j = B_nu(T_j) = c1 nu^3 t / (1 - t), t = e^{-hc nu / kT_j}      (Eq. 2)
// Short characteristics with a linear source (Eqs. 4-7): layer l adds
//   beta_l S_l + gamma_l S_{l+1},  beta = 1 - q, gamma = q - e^{-D},
//   q = (1 - e^{-D}) / D,  D = dtau_l / mu,
// to the intensity entering it from below, with B(T_L) entering the bottom.
// Unrolling that recursion and collecting the terms of each S gives the same
// emergent intensity as a telescoped sum over layers:
//   I_0(mu) = S_0 + mu sum_l (E_l - E_{l+1}) (S_{l+1} - S_l) / dtau_l,
//   E_l = e^{-tau_l / mu}, tau_l the optical depth of level l from the top,
// i.e. the formal solution (Eq. 1) integrated by parts for a piecewise-
// linear source.  Each E_l comes directly from the cumulative tau_l, so the
// small bias of the hardware exponential cannot compound over the layers.
// For optically thin layers (D < kThinLin) the difference is taken as
//   E_l - E_{l+1} = E_l (D - D^2/2 + D^3/6)   (no cancellation),
// chosen per point without a branch.
//   F+ = 2 pi sum_k w_k mu_k I_0(mu_k)                             (Eq. 8)
__device__ __forceinline__ v2 ldf2(const float* p) {
  return __ldg(reinterpret_cast<const unsigned long long*>(p));
}
// a pair of columns of the level-gridded operand: value and T difference
struct __align__(16) RowDiff {
  v2 g, dg;
};
// the last 16 bytes of a LevRecC before its cell index
struct __align__(16) RecTail {
  v2 dtc;
  float upl, rnu;
};
__device__ __forceinline__ RowDiff lds_rd(const float* p) { return *reinterpret_cast<const RowDiff*>(p); }
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

// ---- per-warp bulk-copy pipeline (Blackwell bulk async copies + mbarrier)
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait on a phase: gives up after `limit` SM clock cycles (the
// context's wait limit, ~1 s by default) and reports it.
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity, long long limit) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity))
    if (clock64() - t0 > limit) return false;
  return true;
}
// least limit of the wait that lets a stage's copies land after a wait gave
// up (~5 ms of SM clock, far beyond a copy's latency): the drain waits as long
// as the context's limit allows, and at least this long
constexpr long long kDrainMinCycles = 10000000ll;
// bytes (multiple of 16) from global src to shared dst (both 16-byte aligned),
// completion counted on bar
__device__ __forceinline__ void bulk_copy(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

// Per-warp shared-memory layout of the cached path:
//   rows[2][K + 2][2 kTileNu] floats, per stage (double-buffered by level
//     parity): one level of one T cell of the operand as it is stored
//     ([row][q][value, T difference], the K absorbers and the two CIA pairs);
//   recs[8][16]: the level records, a ring of eight (level j in slot j & 7),
//     filled four at a time;
//   bar[2]: one mbarrier per stage.
struct WarpPipe {
  float* rows;
  float* recs;
  unsigned long long* bar;
};
constexpr int kRecRing = 8;
__host__ __device__ __forceinline__ size_t warp_rows_floats(int max_k, int stages) {
  return (size_t)stages * (2 * max_k + 4) * kTileNu;
}
__host__ __device__ __forceinline__ size_t warp_pipe_bytes(int max_k, int stages) {
  return warp_rows_floats(max_k, stages) * sizeof(float) + kRecRing * sizeof(LevRec) + 2 * sizeof(unsigned long long);
}
__device__ __forceinline__ WarpPipe warp_pipe(unsigned char* base, int max_k, int stages) {
  WarpPipe w;
  w.rows = reinterpret_cast<float*>(base);
  w.recs = reinterpret_cast<float*>(base + warp_rows_floats(max_k, stages) * sizeof(float));
  w.bar = reinterpret_cast<unsigned long long*>(base + warp_rows_floats(max_k, stages) * sizeof(float) +
                                                kRecRing * sizeof(LevRec));
  return w;
}

// First fill of a stage for an item: the operand block of level 0 (T cell
// acell, (K + 2) x 2 kTileNu floats) and the records of levels 0 .. n_rec-1
// into ring slots 0 .. n_rec-1, counted on the stage's barrier.  One lane
// issues everything.  tx_extra (0 except under the context's wait-fault test
// hook) arms the barrier for bytes that never arrive, so that its bounded
// wait runs out.
__device__ __forceinline__ void issue_first(const WarpPipe& w, int st, int K, const float* src_rows, const LevRec* rec,
                                            int n_rec, int lane, unsigned tx_extra) {
  if (lane == 0) {
    const unsigned rows_bytes = (unsigned)((K + 2) * 2 * kTileNu * sizeof(float));
    const unsigned rec_bytes = (unsigned)(n_rec * sizeof(LevRec));
    unsigned long long* bar = w.bar + st;
    mbar_expect_tx(bar, rows_bytes + rec_bytes + tx_extra);
    bulk_copy(w.rows + (size_t)st * (2 * K + 4) * kTileNu, src_rows, rows_bytes, bar);
    bulk_copy(w.recs, rec, rec_bytes, bar);
  }
}

// The in-sweep refill of a stage as straight-line code: every lane runs it,
// and only where `on` (lane 0, a level left to fetch) do the predicated
// instructions arm the stage's barrier with `bytes` and issue the copies
// (the operand block, and records if do_rec), so the sweep has no branch
// around them.
__device__ __forceinline__ void issue_level_pred(unsigned long long* bar, unsigned bytes, bool on, float* dst_rows,
                                                 const float* src_rows, unsigned rows_bytes, float* dst_rec,
                                                 const LevRec* src_rec, unsigned rec_bytes, bool do_rec) {
  asm volatile(
      "{\n"
      " .reg .pred pon, prc;\n"
      " setp.ne.b32 pon, %0, 0;\n"
      " setp.ne.and.b32 prc, %1, 0, pon;\n"
      " @pon mbarrier.arrive.expect_tx.shared::cta.b64 _, [%2], %3;\n"
      " @pon cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%4], [%5], %6, [%2];\n"
      " @prc cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%7], [%8], %9, [%2];\n"
      "}\n" ::"r"((int)on),
      "r"((int)do_rec), "r"(smem_u32(bar)), "r"(bytes), "r"(smem_u32(dst_rows)), "l"(src_rows), "r"(rows_bytes),
      "r"(smem_u32(dst_rec)), "l"(src_rec), "r"(rec_bytes)
      : "memory");
}

// Absorption per molecule from a T-interpolated operand value: 2^x on the
// log10 option (the operand holds log2 of the offset cross-section), x
// itself on the linear option (the operand holds the cross-section).
template <bool LIN>
__device__ __forceinline__ v2 row_value(v2 x) {
  if constexpr (LIN) return x;
  else return ex2_2(x);
}

// Each lane carries kPairs packed pairs of neighbouring wavenumbers: pair p
// holds tile columns 64 p + 2 lane and 64 p + 2 lane + 1, so that a warp's
// shared-memory row reads stay contiguous and every per-level cost that does
// not depend on the wavenumber (records, weights, copies, votes, loop
// control) is paid once for all of them.
constexpr int kPairs = kTileNu / 64;

// Per-lane constants of the wavenumber grid, one set per pair.
struct NuConst {
  float nu0[kPairs], nl0[kPairs], ratio[kPairs];  // first point (head, tail), nu_1 / nu_0
  v2 c1n[kPairs];                                 // c1 nu^3 of both points
};

// Level sweep state of one pair: chi and S of the level above and the
// cumulative optical depth tau_j; for the parabolic source also the slope
// dS/dtau and the optical depth of the layer above.
struct LevelState {
  v2 chip, Sp, tau, dup, dtp;
};

// Accumulators of the emergent flux per pair: one for the linear source
// (every angle node's share folded in), one per node for the parabolic one.
template <int NMU, bool PARA>
struct FluxAcc {
  static constexpr int N = PARA ? NMU : 1;
};

// Physics of one level for the lane's wavenumbers, given chi_j: the Planck
// source, and the layer above it added to the telescoped sum.  SX: some
// level of this sample may have h c nu / k T < 0.0625 on this tile, where
// e^{x} - 1 of the Planck function needs its series (decided per item).
template <int NMU, bool PARA, bool SX, bool ONE>
__device__ __forceinline__ void level_physics(int j, const v2 (&chi)[kPairs], const float upl, const float rnu,
                                              const float r64, const v2 half_dp, const v2 dtc, v2& hdp_prev,
                                              const NuConst& nc, const float thin_dtau, const v2* sMnl,
                                              const v2* sImu, const v2* sMu, const FwdArgs& a, int gs,
                                              v2 (&acc)[kPairs][FluxAcc<NMU, PARA>::N], v2 (&E)[kPairs][NMU],
                                              LevelState (&st)[kPairs]) {
  const float kLn2f = 0.6931471805599453f;
  const v2 one = pk(1.f);
  // Planck source S = c1 nu^3 / (e^x - 1), x = hc nu / kT.  e^x at pair 0's
  // first point is 2^(upl nu) from the FP32 product (relative error of x
  // ~2e-7: e^x to ~2e-7 x); its neighbour is that times e^{hc dnu/kT}, and
  // each further pair 64 points up the previous one times e^{64 hc dnu/kT}.
  // Past FP32's range (x > 88) e^x is +inf and S = c1 nu^3 * 0 = 0, where the
  // true S is below FP32's normal range anyway.  hc nu / kT is smallest at
  // pair 0's first point, which decides whether the small-x form is needed
  // anywhere in the warp.
  v2 Sj[kPairs];
  bool small_x = false;
  if constexpr (SX) small_x = __any_sync(0xffffffffu, upl * nc.nu0[0] * kLn2f < 0.0625f);
  const float z00 = ex2f(upl * nc.nu0[0]);
  v2 z = pk(z00, z00 * rnu);
  const v2 r64p = pk(r64);
#pragma unroll
  for (int p = 0; p < kPairs; ++p) {
    if (p > 0) z = mul2(z, r64p);
    v2 em = sub2(z, one);
    if (SX && small_x) {
      // e^x - 1 without cancellation for small x: x (1 + x/2 + x^2/6 + x^3/24)
      const float x0 = upl * nc.nu0[p] * kLn2f;
      const v2 x = pk(x0, x0 * nc.ratio[p]);
      const v2 ser = mul2(x, fma2(x, fma2(x, fma2(x, pk(1.f / 24.f), pk(1.f / 6.f)), pk(0.5f)), one));
      const float2 xf = up(x), sf = up(ser), of = up(em);
      em = pk(xf.x < 0.0625f ? sf.x : of.x, xf.y < 0.0625f ? sf.y : of.y);
    }
    Sj[p] = mul2(nc.c1n[p], rcp_2(em));
  }
  if constexpr (!PARA) {
    // Linear source, layer j-1 between levels j-1 (top, S_{j-1}) and j
    // (bottom, S_j): it adds (E_{j-1} - E_j) (S_j - S_{j-1}) / dtau to mu's
    // sum, with E_{j-1} - E_j = E_{j-1} (1 - e^{-D}), D = dtau / mu.
    // (S_j - S_{j-1}) / dtau is shared by the nodes.  Where D < kThinLin,
    // 1 - e^{-D} is the polynomial D (1 - D/2 + D^2/6), chosen per point
    // without a branch.  Level 0 enters the same way as a layer of optical depth
    // kTinyTau below a zero source (nothing above it has been added yet):
    // it adds S_0 / mu, the S_0 term of I_0 = S_0 + mu sum_l ...
    // F+ = sum_k 2 pi w_k mu_k I_0(mu_k) = sum_k (2 pi w_k mu_k^2) sum_l ...:
    // each node's E carries its factor 2 pi w_k mu_k^2 in the exponent
    // (E_j = 2^(log2 e (-tau_j / mu_k) + log2(2 pi w_k mu_k^2))), so the nodes'
    // terms of a layer add up before the one multiplication by the shared
    // slope, into one accumulator that ends as F+ itself.  Nodes beyond the
    // setup's count are padded with mu = 1 and a factor 2^-10000 = 0.
    (void)thin_dtau;
    (void)sMnl;
    (void)sImu;
    (void)sMu;
    // st.tau holds -log2(e) tau_j
    v2 dt[kPairs], rdS[kPairs], sum[kPairs];
#pragma unroll
    for (int p = 0; p < kPairs; ++p) {
      // gas trapezoid + gray cloud + kTinyTau
      dt[p] = fma2(hdp_prev, add2(chi[p], st[p].chip), dtc);
      rdS[p] = mul2(sub2(Sj[p], st[p].Sp), rcp_2(dt[p]));
      st[p].tau = fma2(dt[p], pk(-kLog2eF), st[p].tau);
    }
    const v2 c2 = pk(-0.5f), c3 = pk(1.f / 6.f);
#pragma unroll
    for (int k = 0; k < NMU; ++k) {
      // 1 / mu_k, log2(2 pi w_k mu_k^2); with a single setup in the launch (ONE)
      // at fixed kernel-parameter offsets, which the arithmetic reads directly
      const int gk = ONE ? 0 : gs;
      const v2 im = a.node_im[gk][k], lw = a.node_lw[gk][k];
#pragma unroll
      for (int p = 0; p < kPairs; ++p) {
        const v2 En = ex2_2(fma2(st[p].tau, im, lw));   // 2 pi w mu^2 e^{-tau_j / mu}
        const v2 D = mul2(dt[p], im);
        const v2 X = sub2(E[p][k], En);
        const v2 Xs = mul2(E[p][k], mul2(D, fma2(D, fma2(D, c3, c2), one)));
        const float2 Df = up(D), xf = up(X), xsf = up(Xs);
        const v2 cc = pk(Df.x < kThinLin ? xsf.x : xf.x, Df.y < kThinLin ? xsf.y : xf.y);
        sum[p] = k == 0 ? cc : add2(sum[p], cc);
        E[p][k] = En;
      }
    }
#pragma unroll
    for (int p = 0; p < kPairs; ++p) acc[p][0] = fma2(sum[p], rdS[p], acc[p][0]);
  } else if (j > 0) {
    (void)gs;
    // layer j-1 between levels j-1 (top, Sp) and j (bottom, Sj)
    v2 dt[kPairs], rr[kPairs], dS[kPairs];
    float dmin = 3.0e38f;
#pragma unroll
    for (int p = 0; p < kPairs; ++p) {
      dt[p] = fma2(hdp_prev, add2(chi[p], st[p].chip), dtc);   // gas trapezoid + gray cloud
      rr[p] = rcp_2(dt[p]);
      dS[p] = sub2(Sj[p], st[p].Sp);
      st[p].tau = add2(st[p].tau, dt[p]);
      const float2 dtf = up(dt[p]);
      dmin = fminf(dmin, fminf(dtf.x, dtf.y));
    }
    const bool thin = __any_sync(0xffffffffu, dmin < thin_dtau);
    // Parabolic source (Sect. 2.1, higher-order interpolant): over layer
    // j-1 the source is the parabola through levels j-2, j-1, j; in
    // vertical optical depth below level j-1 it is S_{j-1} + c1 t + c2 t^2
    // (divided differences; the top layer keeps c2 = 0), along the ray
    // t -> mu t.  The layer adds E_{j-1} [S_{j-1} M0 + mu c1 M1 + mu^2 c2 M2]
    // with M_k = int_0^D t^k e^{-t} dt, D = dtau / mu, taken from
    //   E M0 = E_{j-1} - E_j, E M1 = E M0 - D E_j, E M2 = 2 E M1 - D^2 E_j,
    // or, where D < kThinD, from the power series of M_k times E_{j-1}.
    // I_0 = sum of the layers + E_L S_L (added after the sweep).
#pragma unroll
    for (int p = 0; p < kPairs; ++p) {
      const v2 du = mul2(dS[p], rr[p]);
      v2 c1 = du, c2 = pk(0.f);
      if (j >= 2) {
        c2 = mul2(sub2(du, st[p].dup), rcp_2(add2(dt[p], st[p].dtp)));
        c1 = sub2(du, mul2(c2, dt[p]));
      }
      st[p].dup = du;
      st[p].dtp = dt[p];
#pragma unroll
      for (int k = 0; k < NMU; ++k) {
        // single setup (ONE): the constants at fixed kernel-parameter offsets
        const v2 mk = ONE ? a.node_mnl0[k] : sMnl[k], im = ONE ? a.node_im[0][k] : sImu[k],
                 mu = ONE ? a.node_mu0[k] : sMu[k];
        const v2 En = ex2_2(mul2(st[p].tau, mk));
        const v2 D = mul2(dt[p], im);
        const v2 D2 = mul2(D, D);
        v2 m0 = sub2(E[p][k], En);
        v2 m1 = sub2(m0, mul2(D, En));
        v2 m2 = sub2(add2(m1, m1), mul2(D2, En));
        if (thin) {
          const v2 Ek = E[p][k];
          const v2 q0 = mul2(D, fma2(D, fma2(D, fma2(D, fma2(D, fma2(D, pk(-1.f / 720.f), pk(1.f / 120.f)),
                                                                pk(-1.f / 24.f)), pk(1.f / 6.f)), pk(-0.5f)), pk(1.f)));
          const v2 q1 = mul2(D2, fma2(D, fma2(D, fma2(D, fma2(D, fma2(D, pk(-1.f / 840.f), pk(1.f / 144.f)),
                                                                 pk(-1.f / 30.f)), pk(1.f / 8.f)), pk(-1.f / 3.f)), pk(0.5f)));
          const v2 q2 = mul2(mul2(D2, D), fma2(D, fma2(D, fma2(D, fma2(D, fma2(D, pk(-1.f / 960.f), pk(1.f / 168.f)),
                                                                          pk(-1.f / 36.f)), pk(0.1f)), pk(-0.25f)),
                                               pk(1.f / 3.f)));
          const v2 s0 = mul2(Ek, q0), s1 = mul2(Ek, q1), s2 = mul2(Ek, q2);
          const float2 Df = up(D), a0 = up(m0), a1 = up(m1), a2 = up(m2), b0 = up(s0), b1 = up(s1), b2 = up(s2);
          const bool tx = Df.x < kThinD, ty = Df.y < kThinD;
          m0 = pk(tx ? b0.x : a0.x, ty ? b0.y : a0.y);
          m1 = pk(tx ? b1.x : a1.x, ty ? b1.y : a1.y);
          m2 = pk(tx ? b2.x : a2.x, ty ? b2.y : a2.y);
        }
        v2 a = fma2(st[p].Sp, m0, acc[p][k]);
        a = fma2(mul2(mu, c1), m1, a);
        acc[p][k] = fma2(mul2(mul2(mu, mu), c2), m2, a);
        E[p][k] = En;
      }
    }
  }
#pragma unroll
  for (int p = 0; p < kPairs; ++p) {
    st[p].chip = chi[p];
    st[p].Sp = Sj[p];
  }
  hdp_prev = half_dp;
}

// Absorption coefficient chi of one level for the lane's pairs (table column
// col of pair 0), read from the FP16 tables in place (the direct path): the
// level record's quarters r0..r2 give the (T, p) corner row, the weights and
// the CIA terms; sA2 / sAc2 the sample's absorber exponents and tails, sPtr
// the absorbers' tables.  log10 sigma is bilinear in (T, log10 p), written as
// corner 00 plus weighted differences (exact partition of unity); two species
// per step, the lane's pairs in parallel; then both CIA pairs.
__device__ __forceinline__ void direct_level_chi(const TablesDev& T, int K, int col, const float4 r0, const float4 r1,
                                                 const float4 r2, const v2* sA2, const v2* sAc2,
                                                 const void* const* sPtr, bool cia0, bool cia1, v2 (&chi)[kPairs]) {
  const int nu_pad = T.nu_pad;
  const unsigned o10 = (unsigned)(T.n_p * nu_pad);
  const __half* __restrict__ ciab0 = T.cia16;
  const __half* __restrict__ ciab1 = T.cia16 + (size_t)T.n_T * nu_pad;
  const v2 L2hi = pk(kL2Hi), L2lo = pk(kL2Lo);
  const v2 wT = pk(r0.y);
  const unsigned rb00 = (unsigned)__float_as_int(r0.x) * (unsigned)nu_pad + (unsigned)col;
  const unsigned rb10 = rb00 + o10, rb01 = rb00 + (unsigned)nu_pad, rb11 = rb10 + (unsigned)nu_pad;
  const v2 wp = pk(r0.z), wq = pk(r0.w);
  v2 chA[kPairs], chB[kPairs];
#pragma unroll
  for (int p = 0; p < kPairs; ++p) chA[p] = chB[p] = pk(0.f);
  for (int s = 0; s < K; s += 2) {
    const bool two = s + 1 < K;
    const __half* b = static_cast<const __half*>(sPtr[s]);
    const __half* c = static_cast<const __half*>(sPtr[two ? s + 1 : s]);
    const v2 A0 = sA2[s], Ac0 = sAc2[s];
    const v2 A1 = sA2[two ? s + 1 : s], Ac1 = two ? sAc2[s + 1] : pk(0.f);
#pragma unroll
    for (int p = 0; p < kPairs; ++p) {
      const unsigned o = 64u * (unsigned)p;
      const v2 f00 = h2f2(ldh2(b + rb00 + o)), f10 = h2f2(ldh2(b + rb10 + o));
      const v2 f01 = h2f2(ldh2(b + rb01 + o)), f11 = h2f2(ldh2(b + rb11 + o));
      const v2 g00 = h2f2(ldh2(c + rb00 + o)), g10 = h2f2(ldh2(c + rb10 + o));
      const v2 g01 = h2f2(ldh2(c + rb01 + o)), g11 = h2f2(ldh2(c + rb11 + o));
      const v2 d01 = sub2(f01, f00), e01 = sub2(g01, g00);
      const v2 d11 = sub2(sub2(f11, f10), d01), e11 = sub2(sub2(g11, g10), e01);
      const v2 l = fma2(wq, d11, fma2(wp, d01, fma2(wT, sub2(f10, f00), f00)));
      const v2 m = fma2(wq, e11, fma2(wp, e01, fma2(wT, sub2(g10, g00), g00)));
      const v2 el = fma2(L2lo, l, fma2(L2hi, l, A0));
      const v2 em = fma2(L2lo, m, fma2(L2hi, m, A1));
      chA[p] = fma2(Ac0, ex2_2(el), chA[p]);
      chB[p] = fma2(Ac1, ex2_2(em), chB[p]);   // zero weight when K is odd and s = K - 1
    }
  }
  if (cia0 || cia1) {
    const unsigned cb = (unsigned)__float_as_int(r2.x) * (unsigned)nu_pad + (unsigned)col;
#pragma unroll
    for (int p = 0; p < kPairs; ++p) {
      const unsigned o = 64u * (unsigned)p;
      if (cia0) {
        const v2 c0 = h2f2(ldh2(ciab0 + cb + o)), c1 = h2f2(ldh2(ciab0 + cb + nu_pad + o));
        const v2 l = fma2(wT, sub2(c1, c0), c0);
        chB[p] = fma2(pk(r2.z), ex2_2(fma2(L2lo, l, fma2(L2hi, l, pk(r1.x)))), chB[p]);
      }
      if (cia1) {
        const v2 c0 = h2f2(ldh2(ciab1 + cb + o)), c1 = h2f2(ldh2(ciab1 + cb + nu_pad + o));
        const v2 l = fma2(wT, sub2(c1, c0), c0);
        chA[p] = fma2(pk(r2.w), ex2_2(fma2(L2lo, l, fma2(L2hi, l, pk(r1.y)))), chA[p]);
      }
    }
  }
#pragma unroll
  for (int p = 0; p < kPairs; ++p) chi[p] = add2(chA[p], chB[p]);
}

// One warp computes one sample on one kTileNu-point wavenumber tile
// (kPairs packed pairs per lane), sweeping the levels from the top (j = 0)
// to the bottom (j = L).  CACHED: absorber rows come from the setup's
// level-gridded operand through the warp's bulk-copy pipeline (rows of level
// j+1 and the record of level j+2 land while level j is computed).
// Otherwise the FP16 tables are read and interpolated bilinearly in place.
template <int NMU, bool CACHED, int KT, bool LIN, bool PARA, bool SX, int ST, bool ONE>
__device__ __forceinline__ void solve_tile(const FwdArgs& a, const SetupDev& S, const TablesDev& T, int i, int tile,
                                           const v2* sA2, const v2* sAc2, const void* const* sPtr,
                                           const v2* sMnl, const v2* sImu, const v2* sMu, int gs,
                                           const WarpPipe& wp_, unsigned& phase_base) {
  const int lane = threadIdx.x & 31;
  if constexpr (HR2_BOUNDS_CHECK) {
    // the item's output row, wavenumber constants, records and table or
    // operand blocks, for every level, checked before anything is read or
    // any copy issued
    bool ok = i >= 0 && i < a.n && S.n_nu <= a.highres_ld && tile >= 0 && tile < S.n_tiles &&
              S.n_lev <= a.rec_ld && S.n_species <= HR2_MAX_SPECIES;
    if constexpr (CACHED) {
      const long long cell_f = (long long)(S.n_species + 2) * 2 * kTileNu;
      const int nTc = T.n_T - 1;
      for (int j = lane; ok && j < S.n_lev; j += 32) {
        const LevRecC r = reinterpret_cast<const LevRecC*>(a.recs + (size_t)i * a.rec_ld)[j];
        ok = S.lvl32 != nullptr && r.acell >= 0 && r.acell < nTc &&
             (long long)r.lvl_off == ((long long)j * nTc + r.acell) * cell_f &&
             (long long)r.lvl_off + cell_f <= S.lvl32_tile_floats;
      }
    } else {
      ok = ok && (long long)(S.tile0 + tile + 1) * kTileNu <= T.nu_pad;
      for (int j = lane; ok && j < S.n_lev; j += 32) {
        const LevRec r = a.recs[(size_t)i * a.rec_ld + j];
        ok = r.acell >= 0 && r.acell <= T.n_T - 2 && r.rowoff >= 0 && r.rowoff / T.n_p == r.acell &&
             r.rowoff % T.n_p <= T.n_p - 2;
      }
      for (int s = 0; s < S.n_species; ++s) ok = ok && S.species[s] >= 0 && S.species[s] < T.n_species;
    }
    if (!bounds_ok(__all_sync(0xffffffffu, ok), lane == 0 ? a.err : nullptr)) return;
  }
  const SampleDev& sd = a.samp[i];
  float* out = a.highres + (size_t)i * a.highres_ld;
  const int col = (S.tile0 + tile) * kTileNu + 2 * lane;  // table column of pair 0's first point
  int kout[kPairs];
  bool in0[kPairs], in1[kPairs];
#pragma unroll
  for (int p = 0; p < kPairs; ++p) {
    kout[p] = col + 64 * p - S.nu_first;
    in0[p] = kout[p] >= 0 && kout[p] < S.n_nu;
    in1[p] = kout[p] + 1 >= 0 && kout[p] + 1 < S.n_nu;
  }
  if (sd.status != 0) {
#pragma unroll
    for (int p = 0; p < kPairs; ++p) {
      if (in0[p]) out[kout[p]] = __int_as_float(0x7fc00000);
      if (in1[p]) out[kout[p] + 1] = __int_as_float(0x7fc00000);
    }
    return;
  }
  NuConst nc;
#pragma unroll
  for (int p = 0; p < kPairs; ++p) {
    const int q = tile * (kTileNu / 2) + lane + 32 * p;   // setup-local pair of columns
    const float4 f = __ldg(&S.nu_pair[q]);
    const float2 c = __ldg(&S.c1n_pair[q]);
    nc.nu0[p] = f.x;    // head
    nc.nl0[p] = f.y;    // tail
    nc.ratio[p] = f.z;
    nc.c1n[p] = pk(c.x, c.y);
  }
  // parabolic source: dtau below which some node is thin (largest mu, padded
  // nodes included), which turns the warp's power-series moments on
  const float thin_dtau = kThinD * S.mu[NMU - 1];
  const int K = S.n_species;
  const int L = S.n_lev - 1;
  const int nT = T.n_T;
  const bool cia0 = T.has_cia[0] != 0, cia1 = T.has_cia[1] != 0;
  const LevRec* __restrict__ rec = a.recs + (size_t)i * a.rec_ld;

  // linear source: E of each node starts at its flux factor 2 pi w mu^2
  // (tau = 0); parabolic: at 1, with one accumulator per node
  v2 acc[kPairs][FluxAcc<NMU, PARA>::N], E[kPairs][NMU];
#pragma unroll
  for (int p = 0; p < kPairs; ++p) {
#pragma unroll
    for (int k = 0; k < FluxAcc<NMU, PARA>::N; ++k) acc[p][k] = pk(0.f);
#pragma unroll
    for (int k = 0; k < NMU; ++k) E[p][k] = PARA ? pk(1.f) : ex2_2(a.node_lw[ONE ? 0 : gs][k]);
  }
  LevelState st[kPairs];
#pragma unroll
  for (int p = 0; p < kPairs; ++p) st[p].chip = st[p].Sp = st[p].tau = st[p].dup = st[p].dtp = pk(0.f);
  v2 hdp_prev = pk(0.f);

  if constexpr (CACHED) {
    // per-sample absorber weights, in registers when the count is fixed
    v2 wreg[KT > 0 ? KT : 1];
    if constexpr (KT > 0) {
#pragma unroll
      for (int q = 0; q < KT; ++q) wreg[q] = sA2[q];
    }
    const v2* sW2 = (KT > 0) ? wreg : sA2;
    // Pipeline over the levels (gph = phase_base + j counts this warp's levels
    // across items).  Record of level j sits in ring slot j & 7.
    //   before the loop: stage of level 0 <- block(0), records 0 .. 7
    //   level j:         wait stage(j)    -> block(j) present
    //                    issue stage(j+1) <- block(j+1) (T cell from record
    //                                        j+1), and where j = 4m >= 4,
    //                                        records j+4 .. j+7
    //                    compute level j
    // (record j+1 is needed at level j; records j+4 .. j+7 land with stage
    // j+1, before level j+3 reads record j+4).  With two stages the refill
    // goes to the other stage before level j is computed; with one stage
    // (more warps per SM fit) it goes to the same stage as soon as level j's
    // opacity has read it, and lands while level j's source and layer run.
    if (phase_base == 0xffffffffu) return;       // this warp's pipeline failed earlier
    const size_t cell_step = (size_t)(K + 2) * 2 * kTileNu;             // one T cell of a level
    const float* lvl_tile = S.lvl32 + (size_t)tile * (L + 1) * (nT - 1) * cell_step;
    const unsigned rows_bytes = (unsigned)(cell_step * sizeof(float));
    const unsigned cia_bytes = (unsigned)(4 * kTileNu * sizeof(float));
    const unsigned ph = phase_base;
    // T cell of the level whose block the stage holds (its CIA rows stay valid
    // for a later level of the same cell); the stage's first fill copies them
    int acell_held = __ldg(&reinterpret_cast<const LevRecC*>(rec)[0].acell);
    // Planck ratio of the current level; each level reads the last quarter of
    // the next record ({T cell, block offset, its ratio}) for the refill and
    // carries the ratio on
    float r64_cur = __ldg(&reinterpret_cast<const LevRecC*>(rec)[0].r64);
    constexpr int kSt = ST;
    issue_first(wp_, kSt == 1 ? 0 : (int)(ph & 1u), K, lvl_tile + (size_t)acell_held * cell_step, rec,
                min(kRecRing, L + 1), lane, a.tx_extra);
    int acell_prev = -1;   // two stages: T cell of the block in the other stage
    // unrolled so that the loop-carried sweep state rotates through register
    // sets instead of being moved back at the end of each level
#pragma unroll 4
    for (int j = 0; j <= L; ++j) {
      const unsigned gph = ph + (unsigned)j;
      // two stages: level gph in stage gph & 1, phase (gph >> 1) & 1 of its
      // barrier; one stage: every level in stage 0, phase gph & 1
      const int stg = kSt == 1 ? 0 : (int)(gph & 1u);
      const unsigned par = kSt == 1 ? (gph & 1u) : ((gph >> 1) & 1u);
      if (!mbar_wait(wp_.bar + stg, par, a.wait_limit)) {
        // the stage never completed: report, drain it (bounded) and stop using
        // this warp's pipeline
        if (lane == 0 && a.err) atomicOr(a.err, kErrWait);
        mbar_wait(wp_.bar + stg, par, max(a.wait_limit, kDrainMinCycles));
        phase_base = 0xffffffffu;
        return;
      }
      __syncwarp();
      // refill a stage with level j+1 and, every fourth level, records
      // j+4 .. j+7: the other stage right away (two stages), or this stage once
      // this level's opacity has read it (one).  Record j+1 gives the block's T
      // cell and its offset in the tile's operand; where the stage already
      // holds that cell's CIA rows (one stage: level j's cell; two: level
      // j-1's, none before this item's first refill) only the absorber rows
      // are copied.
      const int4 q3n = *reinterpret_cast<const int4*>(wp_.recs + ((j + 1) & (kRecRing - 1)) * 16 + kRecCAcell);
      auto refill = [&]() {
        const bool more = j < L;
        const int2 nx = more ? make_int2(q3n.x, q3n.y) : make_int2(0, 0);
        const int sn = kSt == 1 ? 0 : (int)((gph + 1u) & 1u);
        const bool do_rec = (j & 3) == 0 && j >= 4 && j + 4 <= L;
        const unsigned rec_bytes = (unsigned)(min(4, max(0, L - j - 3)) * (int)sizeof(LevRec));
        const int held = kSt == 1 ? acell_held : acell_prev;
        const unsigned rb = held == nx.x ? rows_bytes - cia_bytes : rows_bytes;
        issue_level_pred(wp_.bar + sn, rb + (do_rec ? rec_bytes : 0u), more && lane == 0,
                         wp_.rows + (size_t)sn * (2 * K + 4) * kTileNu, lvl_tile + nx.y, rb,
                         wp_.recs + (size_t)((j + 4) & (kRecRing - 1)) * 16, rec + (j + 4), rec_bytes, do_rec);
        if (kSt == 1) {
          acell_held = nx.x;
        } else {
          acell_prev = acell_held;
          acell_held = nx.x;
        }
      };
      if constexpr (kSt == 2) refill();
      // record j (LevRecC): {wT, wT, wh2h2, wh2h2}, {wh2he, wh2he, half_dp,
      // half_dp}, {dtc, dtc, upl, rnu}, {acell, lvl_off, r64, -}
      const float* rj = wp_.recs + (j & (kRecRing - 1)) * 16;
      const RowDiff rq0 = lds_rd(rj), rq1 = lds_rd(rj + 4);
      const RecTail rq2 = *reinterpret_cast<const RecTail*>(rj + 8);
      const float r64 = r64_cur;
      r64_cur = __int_as_float(q3n.z);
      const v2 wT = rq0.g;
      // stage: [s][q][row, T difference] for pairs q of columns; lane l's
      // pair p is q = l + 32 p
      const float* rows = wp_.rows + (size_t)stg * (2 * K + 4) * kTileNu + 4 * lane;
      // chi = sum_s W_s 2^(log2 10 * log10 sigma_s), W_s = x_s c 10^off_s 2^-shift
      v2 chA[kPairs], chB[kPairs];
#pragma unroll
      for (int p = 0; p < kPairs; ++p) chA[p] = chB[p] = pk(0.f);
      if constexpr (KT > 0) {
        // the item's setup has at most KT absorbers; a padded absorber has
        // weight 0 and reads finite values of the stage (the CIA rows that
        // follow, or the other stage, both initialised)
#pragma unroll
        for (int s = 0; s < KT; s += 2) {
          const v2 w0 = sW2[s], w1 = sW2[s + 1];
#pragma unroll
          for (int p = 0; p < kPairs; ++p) {
            const RowDiff x = lds_rd(rows + s * 2 * kTileNu + 128 * p);
            const RowDiff y = lds_rd(rows + (s + 1) * 2 * kTileNu + 128 * p);
            chA[p] = fma2(w0, row_value<LIN>(fma2(wT, x.dg, x.g)), chA[p]);
            chB[p] = fma2(w1, row_value<LIN>(fma2(wT, y.dg, y.g)), chB[p]);
          }
        }
      } else {
      int s = 0;
      for (; s + 1 < K; s += 2) {
        const v2 w0 = sW2[s], w1 = sW2[s + 1];
#pragma unroll
        for (int p = 0; p < kPairs; ++p) {
          const RowDiff x = lds_rd(rows + s * 2 * kTileNu + 128 * p);
          const RowDiff y = lds_rd(rows + (s + 1) * 2 * kTileNu + 128 * p);
          chA[p] = fma2(w0, row_value<LIN>(fma2(wT, x.dg, x.g)), chA[p]);
          chB[p] = fma2(w1, row_value<LIN>(fma2(wT, y.dg, y.g)), chB[p]);
        }
      }
      if (s < K) {
        const v2 w0 = sW2[s];
#pragma unroll
        for (int p = 0; p < kPairs; ++p) {
          const RowDiff x = lds_rd(rows + s * 2 * kTileNu + 128 * p);
          chA[p] = fma2(w0, row_value<LIN>(fma2(wT, x.dg, x.g)), chA[p]);
        }
      }
      }
      // CIA pair 0, then pair 1; an absent pair has weight 0 and zero rows in
      // the operand (the stage holds finite values for it either way)
      const float* ca = rows + (size_t)2 * K * kTileNu;
      {
        const v2 w0 = rq0.dg, w1 = rq1.g;
#pragma unroll
        for (int p = 0; p < kPairs; ++p) {
          const RowDiff x = lds_rd(ca + 128 * p);
          const RowDiff y = lds_rd(ca + 2 * kTileNu + 128 * p);
          chB[p] = fma2(w0, row_value<LIN>(fma2(wT, x.dg, x.g)), chB[p]);
          chA[p] = fma2(w1, row_value<LIN>(fma2(wT, y.dg, y.g)), chA[p]);
        }
      }
      v2 chi[kPairs];
#pragma unroll
      for (int p = 0; p < kPairs; ++p) chi[p] = add2(chA[p], chB[p]);
      if constexpr (kSt == 1) {
        __syncwarp();   // every lane has read the stage
        refill();
      }
      level_physics<NMU, PARA, SX, ONE>(j, chi, rq2.upl, rq2.rnu, r64, rq1.dg, rq2.dtc, hdp_prev, nc, thin_dtau, sMnl,
                                   sImu, sMu, a, gs, acc, E, st);
      // two stages: every lane is done with stage stg before the next level
      // refills it (one stage: the refill already followed the sync above)
      if constexpr (kSt == 2) __syncwarp();
    }
    phase_base = ph + (unsigned)(L + 1);
  } else {
    const float4* rp = reinterpret_cast<const float4*>(rec);
    // the two-pass path (small batches): the absorption coefficients of every
    // level were computed by k_chi_direct with the same arithmetic
    const float* chi_in = a.chi ? a.chi + (size_t)i * a.rec_ld * a.chi_ld + (size_t)tile * kTileNu + 2 * lane
                                : nullptr;
    for (int j = 0; j <= L; ++j) {
      const float4* q = rp + 4 * j;
      const float4 r0 = __ldg(q), r1 = __ldg(q + 1), r2 = __ldg(q + 2), r3 = __ldg(q + 3);
      v2 chi[kPairs];
      if (chi_in) {
#pragma unroll
        for (int p = 0; p < kPairs; ++p) chi[p] = ldf2(chi_in + (size_t)j * a.chi_ld + 64 * p);
      } else {
        direct_level_chi(T, K, col, r0, r1, r2, sA2, sAc2, sPtr, cia0, cia1, chi);
      }
      level_physics<NMU, PARA, SX, ONE>(j, chi, r1.z, r3.x, r2.y, pk(r1.w), pk(r3.w), hdp_prev, nc, thin_dtau, sMnl,
                                   sImu, sMu, a, gs, acc, E, st);
    }
  }
  // Linear source: the accumulator is F+ (the nodes' flux factors folded
  // in).  Parabolic source: I_0(mu_k) = acc_k + E_L S_L and
  // F+ = sum_k 2 pi w_k mu_k I_0(mu_k).
#pragma unroll
  for (int p = 0; p < kPairs; ++p) {
    float F0 = 0.f, F1 = 0.f;
    if constexpr (PARA) {
      const float2 sL = up(st[p].Sp);
#pragma unroll
      for (int k = 0; k < NMU; ++k) {
        const float2 f = up(acc[p][k]);
        const float wk = S.wflux[k];
        const float2 e = up(E[p][k]);
        F0 = fmaf(wk, fmaf(e.x, sL.x, f.x), F0);
        F1 = fmaf(wk, fmaf(e.y, sL.y, f.y), F1);
      }
    } else {
      const float2 f = up(acc[p][0]);
      F0 = f.x;
      F1 = f.y;
    }
    if (in0[p]) out[kout[p]] = F0;
    if (in1[p]) out[kout[p] + 1] = F1;
  }
}

// Whether some level of sample i has h c nu / k T_j < 0.0625 at the first
// point of the tile (the smallest wavenumber the warp sees), i.e. whether the
// Planck function may need its small-x form anywhere in the sweep.  The
// same test as the per-level one inside the sweep, taken once per item over
// all levels (warp-uniform).
__device__ __forceinline__ bool item_small_x(const FwdArgs& a, const SetupDev& S, const TablesDev& T, int i, int tile) {
  const int lane = threadIdx.x & 31;
  const LevRec* rec = a.recs + (size_t)i * a.rec_ld;
  const float nu_min = (float)(T.nu0 + (double)((S.tile0 + tile) * kTileNu) * T.dnu);
  bool f = false;
  const float* r = reinterpret_cast<const float*>(rec);
  const int o = S.cached ? kRecCUpl : (int)(offsetof(LevRec, upl) / sizeof(float));
  for (int j = lane; j < S.n_lev; j += 32) f |= (__ldg(r + 16 * j + o) * nu_min) * 0.6931471805599453f < 0.0625f;
  return __any_sync(0xffffffffu, f);
}

template <int NMU, bool CACHED, int KT, bool LIN, bool PARA, int ST, bool ONE>
__global__ void __launch_bounds__(kForwardMaxThreads, (CACHED && NMU <= 4 && !PARA) ? kForwardMinBlocksSmall
                                                                                     : kForwardMinBlocks)
    k_forward32(FwdArgs a, int max_k) {
  extern __shared__ __align__(16) unsigned char dyn_smem[];   // cached path: per-warp pipelines
  __shared__ int s_item;
  __shared__ const void* sPtr[HR2_MAX_SPECIES];
  __shared__ v2 sMnl[NMU], sImu[NMU], sMu[NMU];
  __shared__ v2 sA2[kMaxWarps][HR2_MAX_SPECIES];
  __shared__ v2 sAc2[kMaxWarps][HR2_MAX_SPECIES];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  WarpPipe wp_{};
  unsigned phase_base = 0;
  if (CACHED) {
    constexpr int kSt = ST;
    wp_ = warp_pipe(dyn_smem + (size_t)warp * warp_pipe_bytes(max_k, kSt), max_k, kSt);
    // zero the stage rows once, so that rows a padded absorber may read are
    // finite before any copy has written them; then order these generic
    // writes before the bulk copies that will overwrite them
    const int nrow = (int)warp_rows_floats(max_k, kSt);
    for (int q = lane; q < nrow; q += 32) wp_.rows[q] = 0.f;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncwarp();
    if (lane == 0) {
      mbar_init(wp_.bar, 1);
      mbar_init(wp_.bar + 1, 1);
      mbar_fence_init();
    }
    __syncwarp();
  }
  const PlanDev* plan = a.plan;
  const int total = plan->total_items;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_item = (int)atomicAdd(a.counter, 1u);
    __syncthreads();
    const int item = s_item;
    if (item >= total) break;
    int pos = 0;
    while (item >= plan->item_start[pos + 1]) ++pos;
    const int g = plan->order[pos];
    const int rem = item - plan->item_start[pos];
    const int nsb = plan->n_sblocks[g];
    // an item covers a.tiles_per_item consecutive tiles of one block of samples
    const int tgrp = rem / nsb;
    const int sb = rem - tgrp * nsb;
    const SetupDev& S = *a.setups[g];
    const TablesDev& T = *S.tables;
    if (!CACHED && threadIdx.x < S.n_species)
      sPtr[threadIdx.x] = T.sig16 + (size_t)S.species[threadIdx.x] * T.n_T * T.n_p * T.nu_pad;
    if (threadIdx.x < NMU) {
      sMnl[threadIdx.x] = pk(S.mu_nlog2e[threadIdx.x]);
      sImu[threadIdx.x] = pk(S.inv_mu[threadIdx.x]);
      sMu[threadIdx.x] = pk(S.mu[threadIdx.x]);
    }
    const int local = sb * a.warps + warp;
    const bool active = local < plan->count[g];
    const int i = active ? a.perm[plan->first[g] + local] : 0;
    if (CACHED) {
      if (lane < HR2_MAX_SPECIES) sA2[warp][lane] = (active && lane < S.n_species) ? pk(a.samp[i].W[lane]) : pk(0.f);
    } else if (active && lane < S.n_species) {
      {
        sA2[warp][lane] = pk(a.samp[i].A[lane]);
        sAc2[warp][lane] = pk(a.samp[i].Ac[lane]);
      }
    }
    __syncthreads();
    if (active) {
      const int t_end = min(S.n_tiles, (tgrp + 1) * a.tiles_per_item);
      for (int tile = tgrp * a.tiles_per_item; tile < t_end; ++tile) {
        const bool sx = item_small_x(a, S, T, i, tile);
        // ONE (a launch with a single setup; chosen by the launcher): the sweep
        // with the node constants at fixed kernel-parameter offsets (g == 0),
        // which the arithmetic reads directly instead of loading them on every
        // level.  A kernel of its own, so that its registers are allocated for
        // this sweep alone.
        // a batch compiled for a bound KT >= 8 holds setups with KT-4 .. KT
        // absorbers: each item runs the sweep compiled for its own setup's
        // even bound, so that a setup pads at most one absorber (the linear
        // source; the parabolic one keeps the batch's bound)
#define HR2_SOLVE1(KB, SXV, ONEV)                                                                                   \
  solve_tile<NMU, CACHED, KB, LIN, PARA, SXV, ST, ONEV>(a, S, T, i, tile, sA2[warp], sAc2[warp], sPtr, sMnl, sImu, sMu, \
                                                       g, wp_, phase_base)
#define HR2_SOLVE(KB)            \
  do {                           \
    if (sx)                      \
      HR2_SOLVE1(KB, true, ONE); \
    else                         \
      HR2_SOLVE1(KB, false, ONE); \
  } while (0)
        if constexpr (KT >= 8 && !PARA) {
          const int kc = (S.n_species + 1) & ~1;
          if (kc <= KT - 4)
            HR2_SOLVE(KT - 4);
          else if (kc <= KT - 2)
            HR2_SOLVE(KT - 2);
          else
            HR2_SOLVE(KT);
        } else {
          HR2_SOLVE(KT);
        }
#undef HR2_SOLVE
#undef HR2_SOLVE1
      }
    }
  }
}


template <int NMU, bool CACHED, int KT, bool LIN, bool PARA = false, int ST = 2, bool ONE = false>
static cudaError_t launch_one(const FwdArgs& a, int grid, int max_k, cudaStream_t s) {
  const size_t smem = CACHED ? forward32_smem_bytes(a.warps, max_k, ST) : 0;
  if (CACHED) {
    // raise the kernel's dynamic shared-memory limit once (to the largest the
    // library ever asks for), so that later launches, also under stream
    // capture, make no attribute call
    static unsigned long long raised = 0;   // one bit per device
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = 1ull << (dev & 63);
    if (!(raised & bit)) {
      e = cudaFuncSetAttribute(k_forward32<NMU, CACHED, KT, LIN, PARA, ST, ONE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)kForwardSmemCap);
      if (e != cudaSuccess) return e;
      raised |= bit;
    }
    if (smem > kForwardSmemCap) return cudaErrorInvalidValue;
  }
  k_forward32<NMU, CACHED, KT, LIN, PARA, ST, ONE><<<grid, 32 * a.warps, smem, s>>>(a, max_k);
  return cudaGetLastError();
}

// cached path, compiled absorber bound KT: the stage variants that exist
// (forward32_stages): one stage for up to 4 nodes, one or two (by the
// caller's choice) for more nodes with KT >= 8, two otherwise
template <int NMU, int KT, bool LIN, int ST>
static cudaError_t launch_cached_st(const FwdArgs& a, int grid, int max_k, cudaStream_t s) {
  // a launch with a single setup takes the kernel with the node constants at
  // fixed offsets (not in the bounds-checked build)
  if constexpr (!HR2_BOUNDS_CHECK) {
    if (a.n_setups == 1) return launch_one<NMU, true, KT, LIN, false, ST, true>(a, grid, max_k, s);
  }
  return launch_one<NMU, true, KT, LIN, false, ST, false>(a, grid, max_k, s);
}

template <int NMU, int KT, bool LIN>
static cudaError_t launch_kt(const FwdArgs& a, int grid, int max_k, int stages, cudaStream_t s) {
  if constexpr (KT == 0) {
    return launch_cached_st<NMU, 0, LIN, 2>(a, grid, max_k, s);
  } else if constexpr (NMU <= 4) {
    return launch_cached_st<NMU, KT, LIN, 1>(a, grid, max_k, s);
  } else if constexpr (KT >= 8) {
    return stages == 1 ? launch_cached_st<NMU, KT, LIN, 1>(a, grid, max_k, s)
                       : launch_cached_st<NMU, KT, LIN, 2>(a, grid, max_k, s);
  } else {
    return launch_cached_st<NMU, KT, LIN, 2>(a, grid, max_k, s);
  }
}

// cached path: absorber bound kt (0 = any mix of absorber counts, else an
// even bound with every setup at kt - 4 .. kt)
template <int NMU, bool LIN>
static cudaError_t launch_cached(const FwdArgs& a, int grid, int max_k, int kt, int stages, cudaStream_t s) {
  switch (kt) {
    case 0: return launch_kt<NMU, 0, LIN>(a, grid, max_k, stages, s);
    case 2: return launch_kt<NMU, 2, LIN>(a, grid, max_k, stages, s);
    case 4: return launch_kt<NMU, 4, LIN>(a, grid, max_k, stages, s);
    case 6: return launch_kt<NMU, 6, LIN>(a, grid, max_k, stages, s);
    case 8: return launch_kt<NMU, 8, LIN>(a, grid, max_k, stages, s);
    case 10: return launch_kt<NMU, 10, LIN>(a, grid, max_k, stages, s);
    case 12: return launch_kt<NMU, 12, LIN>(a, grid, max_k, stages, s);
    case 14: return launch_kt<NMU, 14, LIN>(a, grid, max_k, stages, s);
    case 16: return launch_kt<NMU, 16, LIN>(a, grid, max_k, stages, s);
    default: return cudaErrorInvalidValue;
  }
}

// parabolic source on the level-gridded path: the same absorber bounds as the
// linear source, two stages
template <int NMU, int KT, bool LIN>
static cudaError_t launch_para_kt(const FwdArgs& a, int grid, int max_k, cudaStream_t s) {
  // a launch with a single setup takes the kernel with the node constants at
  // fixed offsets (not in the bounds-checked build)
  if constexpr (!HR2_BOUNDS_CHECK) {
    if (a.n_setups == 1) return launch_one<NMU, true, KT, LIN, true, 2, true>(a, grid, max_k, s);
  }
  return launch_one<NMU, true, KT, LIN, true, 2, false>(a, grid, max_k, s);
}

template <int NMU, bool LIN>
static cudaError_t launch_para(const FwdArgs& a, int grid, int max_k, int kt, cudaStream_t s) {
  switch (kt) {
    case 0: return launch_para_kt<NMU, 0, LIN>(a, grid, max_k, s);
    case 2: return launch_para_kt<NMU, 2, LIN>(a, grid, max_k, s);
    case 4: return launch_para_kt<NMU, 4, LIN>(a, grid, max_k, s);
    case 6: return launch_para_kt<NMU, 6, LIN>(a, grid, max_k, s);
    case 8: return launch_para_kt<NMU, 8, LIN>(a, grid, max_k, s);
    case 10: return launch_para_kt<NMU, 10, LIN>(a, grid, max_k, s);
    case 12: return launch_para_kt<NMU, 12, LIN>(a, grid, max_k, s);
    case 14: return launch_para_kt<NMU, 14, LIN>(a, grid, max_k, s);
    case 16: return launch_para_kt<NMU, 16, LIN>(a, grid, max_k, s);
    default: return cudaErrorInvalidValue;
  }
}

template <int NMU>
static cudaError_t launch_nmu(const FwdArgs& a, int grid, bool cached, bool linear, bool para, int max_k, int kt,
                              int stages, cudaStream_t s) {
  if (para) {
    if (!cached) return linear ? cudaErrorInvalidValue : launch_one<NMU, false, 0, false, true>(a, grid, max_k, s);
    return linear ? launch_para<NMU, true>(a, grid, max_k, kt, s) : launch_para<NMU, false>(a, grid, max_k, kt, s);
  }
  if (!cached) return linear ? cudaErrorInvalidValue : launch_one<NMU, false, 0, false>(a, grid, max_k, s);
  return linear ? launch_cached<NMU, true>(a, grid, max_k, kt, stages, s)
                : launch_cached<NMU, false>(a, grid, max_k, kt, stages, s);
}

}  // namespace hr2
