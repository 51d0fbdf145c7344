// pf_kernels.cu -- sm_103a kernels of the bootstrap particle filter
// (arXiv 1306.3277, Algorithm 2) and their host-side launchers.
//
// One step i of one filter is two launches over its tiles of TILE particles,
// chained by programmatic dependent launch:
//   k_propagate  gather x(t_{i-1}) at the ancestors, propagate to t_i (the
//                windkessel's Euler or exact transition, Lorenz '96 RK4
//                substeps with additive or in-step Wiener noise), weight with
//                y(t_i) in FP64 (skipped at a step without an observation),
//                then per tile the max, the inclusive prefix of
//                exp(ell - M_tile) (exp_weight: double-float on the FP32
//                unit; for the small states the prefix is an exact
//                fixed-point integer scan rounded once to FP64) and its
//                total.  The last tile of each
//                group of GROUP tiles combines the group; the last group
//                combines the filter: max, scaled sums, likelihood increment,
//                ESS test, resampling uniform.
//   k_resample   per tile: cumulative weights C_k = base + scale * prefix,
//                each particle's count of targets below C_k (systematic,
//                stratified or multinomial), and each particle's offspring
//                range written out by its thread, its warp or its block.
// The multinomial scheme adds three small kernels between the two (its
// sorted targets); the path sample adds a pick, a trace and a copy kernel.
// Small filters of a batch may instead run whole, each on one thread-block
// cluster (k_filter_cluster), through the same per-tile functions.
// Any number of filters share a launch: the tile map lists (filter, tile)
// pairs, and every reduction is per tile / group / filter in a fixed order,
// so a filter's result does not depend on what else is in the launch.
#include <algorithm>
#include <cmath>
#include <cstdio>

#include "pf_dev.cuh"
#include "pf_internal.h"

namespace pfb {

static_assert(TILE == GROUP, "the group combine maps one tile partial per thread");

__device__ __forceinline__ double fmaR(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fmaR(float a, float b, float c) { return fmaf(a, b, c); }

// One classic RK4 step of dt for dx_n/dt = (x_{n+1} - x_{n-2}) x_{n-1} - x_n + F
// (cyclic), the right-hand side evaluated as fma(x_{n+1} - x_{n-2}, x_{n-1}, F - x_n)
// and the update accumulated as x + h/6 k1 + h/3 k2 + h/3 k3 + h/6 k4.
// force(n) is the forcing of component n: F, or F plus the substep's Wiener
// increment over its length for the stochastic form.
template <int N, typename R, typename Force>
__device__ __forceinline__ void l96_rk4_step_f(R (&x)[N], Force force, R dt, R h2, R h3, R h6) {
  R acc[N], xa[N], xb[N];
#pragma unroll
  for (int n = 0; n < N; ++n) {
    const R k = fmaR(x[(n + 1) % N] - x[(n + N - 2) % N], x[(n + N - 1) % N], force(n) - x[n]);
    acc[n] = fmaR(h6, k, x[n]);
    xa[n] = fmaR(h2, k, x[n]);
  }
#pragma unroll
  for (int n = 0; n < N; ++n) {
    const R k = fmaR(xa[(n + 1) % N] - xa[(n + N - 2) % N], xa[(n + N - 1) % N], force(n) - xa[n]);
    acc[n] = fmaR(h3, k, acc[n]);
    xb[n] = fmaR(h2, k, x[n]);
  }
#pragma unroll
  for (int n = 0; n < N; ++n) {
    const R k = fmaR(xb[(n + 1) % N] - xb[(n + N - 2) % N], xb[(n + N - 1) % N], force(n) - xb[n]);
    acc[n] = fmaR(h3, k, acc[n]);
    xa[n] = fmaR(dt, k, x[n]);
  }
#pragma unroll
  for (int n = 0; n < N; ++n) {
    const R k = fmaR(xa[(n + 1) % N] - xa[(n + N - 2) % N], xa[(n + N - 1) % N], force(n) - xa[n]);
    x[n] = fmaR(h6, k, acc[n]);
  }
}

template <int N, typename R>
__device__ __forceinline__ void l96_rk4_step(R (&x)[N], R F, R dt, R h2, R h3, R h6) {
  l96_rk4_step_f<N, R>(x, [F](int) { return F; }, dt, h2, h3, h6);
}

// Lorenz '96 right-hand side for the component pair p = (p, p + H) of a state
// stored as H = N/2 pairs; the cyclic neighbours of the first and last pairs
// are the swapped halves of the pairs at the other end.
template <int H>
__device__ __forceinline__ f32x2 l96_rhs2(const f32x2 (&Y)[H], int p, f32x2 FF) {
  const f32x2 xp1 = p + 1 < H ? Y[(p + 1) % H] : swp(Y[0]);
  const f32x2 xm2 = p >= 2 ? Y[(p + H - 2) % H] : swp(Y[(p + H - 2) % H]);
  const f32x2 xm1 = p >= 1 ? Y[(p + H - 1) % H] : swp(Y[H - 1]);
  return fma2(sub2(xp1, xm2), xm1, sub2(FF, Y[p]));
}

// The RK4 step of l96_rk4_step_f on the packed state (same operations per
// lane); force(p) is the packed forcing of the pair p.
template <int H, typename Force>
__device__ __forceinline__ void l96_rk4_step2_f(f32x2 (&X)[H], Force force, f32x2 dt, f32x2 h2,
                                                f32x2 h3, f32x2 h6) {
  f32x2 acc[H], A[H], B[H];
#pragma unroll
  for (int p = 0; p < H; ++p) {
    const f32x2 k = l96_rhs2<H>(X, p, force(p));
    acc[p] = fma2(h6, k, X[p]);
    A[p] = fma2(h2, k, X[p]);
  }
#pragma unroll
  for (int p = 0; p < H; ++p) {
    const f32x2 k = l96_rhs2<H>(A, p, force(p));
    acc[p] = fma2(h3, k, acc[p]);
    B[p] = fma2(h2, k, X[p]);
  }
#pragma unroll
  for (int p = 0; p < H; ++p) {
    const f32x2 k = l96_rhs2<H>(B, p, force(p));
    acc[p] = fma2(h3, k, acc[p]);
    A[p] = fma2(dt, k, X[p]);
  }
#pragma unroll
  for (int p = 0; p < H; ++p) {
    const f32x2 k = l96_rhs2<H>(A, p, force(p));
    X[p] = fma2(h6, k, acc[p]);
  }
}

template <int H>
__device__ __forceinline__ void l96_rk4_step2(f32x2 (&X)[H], f32x2 FF, f32x2 dt, f32x2 h2,
                                              f32x2 h3, f32x2 h6) {
  l96_rk4_step2_f<H>(X, [FF](int) { return FF; }, dt, h2, h3, h6);
}

// Normals number 0..N-1 of the stream (j, i, purpose) into z (N a multiple of 4
// for Lorenz '96; the windkessel uses its own loop).
template <int N>
__device__ __forceinline__ void normals(double (&z)[N], uint64_t seed, uint32_t j, uint32_t i,
                                        uint32_t purpose, uint32_t b0 = 0) {
#pragma unroll
  for (int b = 0; b < (N + 1) / 2; ++b) {
    double z0, z1;
    normal_pair64(rng_block(seed, j, i, purpose, b0 + b), &z0, &z1);
    z[2 * b] = z0;
    if (2 * b + 1 < N) z[2 * b + 1] = z1;
  }
}
template <int N>
__device__ __forceinline__ void normals(float (&z)[N], uint64_t seed, uint32_t j, uint32_t i,
                                        uint32_t purpose, uint32_t b0 = 0) {
#pragma unroll
  for (int b = 0; b < (N + 3) / 4; ++b) {
    const uint4 w = rng_block(seed, j, i, purpose, b0 + b);
    float z0, z1, z2, z3;
    normal_pair32(w.x, w.y, &z0, &z1);
    normal_pair32(w.z, w.w, &z2, &z3);
    z[4 * b] = z0;
    if (4 * b + 1 < N) z[4 * b + 1] = z1;
    if (4 * b + 2 < N) z[4 * b + 2] = z2;
    if (4 * b + 3 < N) z[4 * b + 3] = z3;
  }
}

__device__ __forceinline__ double to_double(double v) { return v; }
// Exact float -> double for finite normal floats built with integer ops
// (rebias the exponent, shift the mantissa), leaving the FP64 unit, which
// B300 runs at 1/64 of the FP32 rate, to the weight arithmetic itself; zero,
// subnormal, infinite and NaN inputs take the ordinary conversion.
__device__ __forceinline__ double to_double(float v) {
  const unsigned b = __float_as_uint(v);
  const unsigned e = b & 0x7f800000u;
  if (e == 0u || e == 0x7f800000u) return double(v);
  const unsigned hi = (b & 0x80000000u) | (((e >> 23) + 896u) << 20) | ((b & 0x007fffffu) >> 3);
  const unsigned lo = (b & 7u) << 29;
  return __hiloint2double(int(hi), int(lo));
}
template <typename R> __device__ __forceinline__ R from_double(double v);
template <> __device__ __forceinline__ double from_double<double>(double v) { return v; }
template <> __device__ __forceinline__ float from_double<float>(double v) { return __double2float_rn(v); }

// Invariant-violation counters of a checked build (see PF_CHECKED).
__device__ unsigned long long g_checks[CHK_KINDS];
__device__ __forceinline__ void check_failed(int kind) { atomicAdd(&g_checks[kind], 1ull); }

// ---------------------------------------------------------------------------
// Weight exponential w = e^d, d = ell - M <= 0, at FP64 accuracy with two
// FP64 operations.  B300's FP64 unit runs at 1/64 of the FP32 rate and the
// library exponential spends about a dozen FP64 instructions per call, which
// made it a fifth of the small-state propagate kernels; here the work runs on
// the FP32 and integer units instead.  Method: Tang's table-driven
// exponential (ACM TOMS 15(2), 1989), d = (256 m + j) ln2/256 + r with
// |r| <= ln2/512, e^d = 2^m 2^(j/256) e^r, evaluated with double-float
// (unevaluated sums of two floats; Dekker 1971, Knuth's two-sum):
//  * d splits exactly into three floats (24 + 24 + 5 significant bits);
//  * k = rint(d 256/ln2) in FP32; r = d - k ln2/256 with ln2/256 in three
//    floats (the first product is exact inside the fma), carried as a
//    double-float;
//  * q = e^r - 1 = r + r^2/2 + (r^3/6 + r^4/24 + r^5/120), the square as a
//    double-float, the cubic tail in FP32;
//  * in FP64: Q = qh + ql, W = T_j (1 + Q) by one fma (T_j = 2^(j/256)
//    rounded to the nearest double), and 2^m goes into W's exponent bits.
// Relative error about 2^-52 (tests compare it with the correctly rounded
// value).  Outside -700 < d <= 0 it takes the library exponential (d > 0,
// d in (-745.2, -700]) or returns 0 (d <= -745.2, including -inf).
// ---------------------------------------------------------------------------
#include "pf_exp2_table.h"

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bp = __fsub_rn(s, a);
  const float ap = __fsub_rn(s, bp);
  e = __fadd_rn(__fsub_rn(a, ap), __fsub_rn(b, bp));
}
__device__ __forceinline__ float pow2f(int e) {  // 2^e for -126 <= e <= 127
  return __uint_as_float(unsigned(e + 127) << 23);
}

__device__ __forceinline__ double exp_weight(double d) {
  const unsigned long long ub = static_cast<unsigned long long>(__double_as_longlong(d));
  if (ub == 0ull) return 1.0;                          // +0
  if (ub < 0x8000000000000000ull) return exp(d);       // d > 0, +inf, +NaN
  if (ub > 0xfff0000000000000ull) return d;            // -NaN
  if (ub >= 0xc08749999999999aull) return 0.0;         // d <= -745.2, -inf
  if (ub >= 0xc085e00000000000ull) return exp(d);      // -745.2 < d <= -700
  const int ex = int((ub >> 52) & 0x7ffu) - 1023;
  if (ex < -60) return 1.0;                            // |d| < 2^-60 (and -0)
  // d = -(mh 2^(ex-23) + mm 2^(ex-47) + ml 2^(ex-52)), each part exact in FP32
  const unsigned long long m = (ub & 0x000fffffffffffffull) | 0x0010000000000000ull;
  const unsigned mh = unsigned(m >> 29), mm = unsigned(m >> 5) & 0xffffffu, ml = unsigned(m) & 31u;
  const float dh = __uint_as_float(0x80000000u | (unsigned(ex + 127) << 23) | (mh & 0x7fffffu));
  const float dm = -__fmul_rn(__uint2float_rn(mm), pow2f(ex - 47));
  const float dl = -__fmul_rn(__uint2float_rn(ml), pow2f(ex - 52));
  // range reduction: |k| < 2^18, r1 = dh - k C1 exact
  const float kf = rintf(__fmul_rn(dh, 0x1.715476p+8f));  // 256 / ln2
  const int k = int(kf);
  constexpr float C1 = 0x1.62e43p-9f, C2 = -0x1.05c61p-37f, C3 = -0x1.950d88p-62f;
  const float r1 = __fmaf_rn(-kf, C1, dh);
  const float p2 = __fmul_rn(kf, C2);
  const float e2 = __fmaf_rn(kf, C2, -p2);  // kf C2 = p2 + e2 exactly
  const float p3 = __fmul_rn(kf, C3);
  float a, ae, b, be, rh, rl;
  two_sum(r1, dm, a, ae);
  two_sum(a, -p2, b, be);
  const float low = __fsub_rn(__fsub_rn(__fadd_rn(__fadd_rn(ae, be), dl), e2), p3);
  two_sum(b, low, rh, rl);  // r = rh + rl
  // q = e^r - 1
  const float sh = __fmul_rn(rh, rh);
  const float sl = __fadd_rn(__fmaf_rn(rh, rh, -sh), __fmul_rn(__fmul_rn(2.0f, rh), rl));
  const float poly = __fmaf_rn(__fmaf_rn(rh, 0x1.111112p-7f, 0x1.555556p-5f), rh, 0x1.555556p-3f);
  const float tail = __fmul_rn(__fmul_rn(sh, rh), poly);
  float u, ue, qh, ql;
  two_sum(rh, __fmul_rn(0.5f, sh), u, ue);
  const float lo = __fadd_rn(__fadd_rn(__fadd_rn(ue, __fmul_rn(0.5f, sl)), rl), tail);
  two_sum(u, lo, qh, ql);
  const double Q = __dadd_rn(to_double(qh), to_double(ql));
  const double T = __ldg(&k_exp2_256[k & 255]);
  const double W = __fma_rn(T, Q, T);  // in [0.998, 2): 2^(k >> 8) W stays a normal number
  return __longlong_as_double(__double_as_longlong(W) + (static_cast<long long>(k >> 8) << 52));
}

// log S of a filter's weight sum S = sum_j e^(ell_j - M) >= 1 (the maximal
// particle contributes e^0 = 1), for the likelihood increment M + log S.  The
// library's FP64 logarithm is a long chain of FP64 operations, which B300 runs
// at 1/64 of the FP32 rate, on the serial path of every step's combine.  Here:
// y0 = logf(S) in FP32 (the library's single-precision logarithm, within one
// FP32 ulp of log S), then one Newton step for e^y = S in FP64,
// t = S e^(-y0) - 1 with the weight exponential (relative error about 2^-52),
// log S = y0 + log1p(t) = y0 + (t - t^2/2).  |t| is about y0's error, at most
// 2^-17 (2^-19 for S <= 2^31), so the omitted t^3/3 stays below 2^-52
// (2^-58).  Absolute error a few units of 2^-53 times max(1, log S) (tests
// compare it with correctly rounded values); seven FP64-pipe operations.
// log 1 = 0 exactly; outside 1 <= S <= 2^120 (never reached by a filter) the
// library logarithm.
__device__ __forceinline__ double log_sum(double S) {
  if (S == 1.0) return 0.0;
  if (!(S > 1.0 && S <= 0x1p120)) return log(S);
  const double y0 = to_double(logf(__double2float_rn(S)));
  const double t = fma(S, exp_weight(-y0), -1.0);
  return y0 + fma(-0.5 * t, t, t);
}

// The combines' exponential and logarithm: the two functions above (OWN), or
// the library's for the large states, whose register-bound propagate kernel
// measurably slows (0.7 %) when their code is compiled into it.  A model class
// uses one choice in every launch form, so every form gives the same bits.
template <bool OWN>
__device__ __forceinline__ double combine_exp(double d) {
  if constexpr (OWN) return exp_weight(d);
  else return exp(d);
}
template <bool OWN>
__device__ __forceinline__ double combine_log(double s) {
  if constexpr (OWN) return log_sum(s);
  else return log(s);
}
template <int KIND, int N>
struct OwnCombineMath {
  static constexpr bool value = !(l96_kind(KIND) && N >= 16);
};
// The in-tile cumulative weights of a model class: the exact fixed-point scan
// (block_scan_fixed) for the small states, whose kernels are bound by the FP64
// unit; the canonical FP64 scan (block_scan) for Lorenz '96 with N >= 16,
// bound by FP32 issue, where the scan's integer work measured slower.  Every
// launch form of a class takes the same one, so its results do not depend on
// the form.
template <int KIND, int N>
struct FixedPrefix {
  static constexpr bool value = !(l96_kind(KIND) && N >= 16);
};

// The systematic resampling uniform of step i: u in [0, 1) from words 1:0 of
// Philox block (0, i, RESAMPLE, 0).
__device__ __forceinline__ double resample_uniform(const FilterDev& fd, int i) {
  const uint4 w = rng_block(fd.seed, 0u, uint32_t(i), PURPOSE_RESAMPLE, 0u);
  return u53_closed_open(w.x, w.y);
}

// The paper's windkessel transition: s steps x <- a x + b (F_k + sd z_mm),
// a = exp(-dt/(RC)) (own exponential), b = R (1 - a), sd = dt sqrt(sigma2),
// z_mm = normal number mm of stream (j, i, PROP); a, b, sd in FP64, rounded to
// the state precision.
// Normal numbers mm and mm + 1 of stream (j, i, PROP) of an FP64 windkessel
// filter: read from its table when they were drawn ahead (k_noise_wk64: the
// same Philox block and Box-Muller pair), else drawn here.
__device__ __forceinline__ void wk_normals64(const FilterDev& fd, uint32_t j, int i, int mm,
                                             double (&z)[2]) {
  if (fd.znoise) {
    const double* zr = fd.znoise + (int64_t(i - 1) * fd.s + mm) * fd.P + j;
    z[0] = zr[0];
    z[1] = mm + 1 < fd.s ? zr[fd.P] : 0.0;
  } else {
    normal_pair64(rng_block(fd.seed, j, uint32_t(i), PURPOSE_PROP, uint32_t(mm >> 1)), &z[0],
                  &z[1]);
  }
}

// The filter's constants (a, b, sd) of the exact windkessel transition, computed
// by one thread per block: an FP64 exponential, a division and a square root
// that every particle shares.
template <typename R>
__device__ __forceinline__ void wkx_constants(const FilterDev& fd, R (&c)[3]) {
  const double Rr = fd.theta[0], Cc = fd.theta[1];
  const double a64 = exp_own(-(fd.dt / (Rr * Cc)));
  c[0] = from_double<R>(a64);
  c[1] = from_double<R>(Rr * (1.0 - a64));
  c[2] = from_double<R>(fd.dt * sqrt(fd.theta[3]));
}

template <typename R>
__device__ __forceinline__ void wkx_propagate(const FilterDev& fd, uint32_t j, int i, R& xv,
                                              const R (&c)[3]) {
  const int s = fd.s;
  const R a = c[0], b = c[1], sd = c[2];
  const double* fl = fd.flow + int64_t(i - 1) * s;
  if constexpr (sizeof(R) == 8) {
    for (int mm = 0; mm < s; mm += 2) {
      double z[2];
      wk_normals64(fd, j, i, mm, z);
#pragma unroll
      for (int e = 0; e < 2; ++e)
        if (mm + e < s) xv = fmaR(a, xv, b * fmaR(sd, R(z[e]), R(fl[mm + e])));
    }
  } else {
    for (int mm = 0; mm < s; mm += 4) {
      const uint4 w = rng_block(fd.seed, j, uint32_t(i), PURPOSE_PROP, uint32_t(mm >> 2));
      float z[4];
      normal_pair32(w.x, w.y, &z[0], &z[1]);
      normal_pair32(w.z, w.w, &z[2], &z[3]);
#pragma unroll
      for (int e = 0; e < 4; ++e)
        if (mm + e < s) xv = fmaR(a, xv, b * fmaR(sd, z[e], from_double<R>(fl[mm + e])));
    }
  }
}

// Windkessel propagation: s Euler substeps x <- x + dt (F_k/C - x/(RC)) +
// sqrt(q) z_mm (normal number mm of stream (j, i, PROP)).  fc, when given,
// holds the step's F_k/C, and kc the filter's sqrt(q), RC, C and dt in R (the
// same operations, made once per block: every particle shares them; in FP64
// the square root is a long chain on B300's 1/64-rate FP64 unit, and in FP32
// the conversions from FP64 run on that unit too).
template <typename R>
__device__ __forceinline__ void wk_propagate(const FilterDev& fd, uint32_t j, int i, R& xv,
                                             const R* fc, const R* kc) {
  const int s = fd.s;
  const R Cc = kc[2];
  const R dt = kc[3];
  const R sq = kc[0];
  const R RC = kc[1];
  const double* fl = fd.flow + int64_t(i - 1) * s;
  if constexpr (sizeof(R) == 8) {
    for (int mm = 0; mm < s; mm += 2) {
      double z[2];
      wk_normals64(fd, j, i, mm, z);
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        if (mm + e < s) {
          const R fkc = fc ? fc[mm + e] : R(fl[mm + e]) / Cc;
          const R drift = fkc - xv / RC;
          xv = fmaR(dt, drift, xv);
          xv = fmaR(sq, R(z[e]), xv);
        }
      }
    }
  } else {
    for (int mm = 0; mm < s; mm += 4) {
      const uint4 w = rng_block(fd.seed, j, uint32_t(i), PURPOSE_PROP, uint32_t(mm >> 2));
      float z[4];
      normal_pair32(w.x, w.y, &z[0], &z[1]);
      normal_pair32(w.z, w.w, &z[2], &z[3]);
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        if (mm + e < s) {
          const R fkc = fc ? fc[mm + e] : from_double<R>(fl[mm + e]) / Cc;
          const R drift = fkc - xv / RC;
          xv = fmaR(dt, drift, xv);
          xv = fmaR(sq, R(z[e]), xv);
        }
      }
    }
  }
}

// Windkessel weight: log N(y; x + Z F(t_i), r) without its constant,
// (y - x - Z F)^2 times cw = -0.5 / r.
template <typename R>
__device__ __forceinline__ double wk_weight(const FilterDev& fd, int i, R xv, double yi,
                                            double cw) {
  const double h = fma(fd.theta[2], fd.flow[int64_t(i) * fd.s], to_double(xv));
  const double d = yi - h;
  const double acc = fma(d, d, 0.0);
  return acc * cw;
}

// The FP32 Lorenz '96 step constants of a run, as l96_propagate derives them
// from theta and dt: F, dt, dt/2, dt/3, dt/6, sqrt(q).  Computed once per run
// into the control block (the conversions from FP64 are FP64-unit work, which
// bounds the small-state kernels) and read back by every block.
__device__ __forceinline__ void l96_constants32(const FilterDev& fd, float* lf) {
  const float dt = __double2float_rn(fd.dt);
  lf[0] = __double2float_rn(fd.theta[0]);
  lf[1] = dt;
  lf[2] = 0.5f * dt;
  lf[3] = dt / 3.0f;
  lf[4] = dt / 6.0f;
  lf[5] = sqrtf(__double2float_rn(fd.theta[1]));
}

// Lorenz '96 propagation: s RK4 substeps, then additive sqrt(q) z_n on every
// component.  In FP32 the state is integrated as N/2 packed pairs (components
// p and p + N/2), which issues half the instructions for the same bits.
template <int N, typename R>
__device__ __forceinline__ void l96_propagate(const FilterDev& fd, uint32_t j, int i, R (&x)[N],
                                              const float* lf = nullptr) {
  // lf (FP32 state only): the run's constants from the control block
  const bool cst = sizeof(R) == 4 && lf != nullptr;
  const R F = cst ? R(lf[0]) : from_double<R>(fd.theta[0]);
  const R dt = cst ? R(lf[1]) : from_double<R>(fd.dt);
  const R h2 = cst ? R(lf[2]) : R(0.5) * dt, h3 = cst ? R(lf[3]) : dt / R(3.0),
          h6 = cst ? R(lf[4]) : dt / R(6.0);
  if constexpr (sizeof(R) == 4 && N % 2 == 0) {
    constexpr int H = N / 2;
    f32x2 X[H];
#pragma unroll
    for (int p = 0; p < H; ++p) X[p] = pk(x[p], x[p + H]);
    const f32x2 FF = pk(F, F), dt2 = pk(dt, dt), h22 = pk(h2, h2), h32 = pk(h3, h3),
                h62 = pk(h6, h6);
    for (int mm = 0; mm < fd.s; ++mm) l96_rk4_step2<H>(X, FF, dt2, h22, h32, h62);
    R z[N];
    normals<N>(z, fd.seed, j, uint32_t(i), PURPOSE_PROP);
    const R sx = cst ? R(lf[5]) : sqrt(from_double<R>(fd.theta[1]));
    const f32x2 sx2 = pk(sx, sx);
#pragma unroll
    for (int p = 0; p < H; ++p) {
      X[p] = fma2(sx2, pk(z[p], z[p + H]), X[p]);
      upk(X[p], x[p], x[p + H]);
    }
  } else {
    for (int mm = 0; mm < fd.s; ++mm) l96_rk4_step<N, R>(x, F, dt, h2, h3, h6);
    R z[N];
    normals<N>(z, fd.seed, j, uint32_t(i), PURPOSE_PROP);
    const R sx = cst ? R(lf[5]) : sqrt(from_double<R>(fd.theta[1]));
#pragma unroll
    for (int n = 0; n < N; ++n) x[n] = fmaR(sx, z[n], x[n]);
  }
}

// The paper's Lorenz '96 transition: s RK4 substeps, substep mm with the
// forcing F + sqrt(q/dt) z_{mm N + n} on component n (the Wiener increment
// over the substep divided by its length), normal numbers mm N .. mm N + N-1
// of stream (j, i, PROP); no noise after the substeps.
template <int N, typename R>
__device__ __forceinline__ void l96w_propagate(const FilterDev& fd, uint32_t j, int i,
                                               R (&x)[N]) {
  const R F = from_double<R>(fd.theta[0]);
  const R dt = from_double<R>(fd.dt);
  const R h2 = R(0.5) * dt, h3 = dt / R(3.0), h6 = dt / R(6.0);
  const R sw = sqrt(from_double<R>(fd.theta[1]) / dt);
  constexpr uint32_t per_block = sizeof(R) == 4 ? 4u : 2u;  // normals per Philox block
  if constexpr (sizeof(R) == 4 && N % 2 == 0) {
    constexpr int H = N / 2;
    f32x2 X[H];
#pragma unroll
    for (int p = 0; p < H; ++p) X[p] = pk(x[p], x[p + H]);
    const f32x2 FF = pk(F, F), dt2 = pk(dt, dt), h22 = pk(h2, h2), h32 = pk(h3, h3),
                h62 = pk(h6, h6), sw2 = pk(sw, sw);
    for (int mm = 0; mm < fd.s; ++mm) {
      R z[N];
      normals<N>(z, fd.seed, j, uint32_t(i), PURPOSE_PROP, uint32_t(mm) * (N / per_block));
      f32x2 FV[H];
#pragma unroll
      for (int p = 0; p < H; ++p) FV[p] = fma2(sw2, pk(z[p], z[p + H]), FF);
      l96_rk4_step2_f<H>(X, [&](int p) { return FV[p]; }, dt2, h22, h32, h62);
    }
#pragma unroll
    for (int p = 0; p < H; ++p) upk(X[p], x[p], x[p + H]);
  } else {
    for (int mm = 0; mm < fd.s; ++mm) {
      R z[N];
      normals<N>(z, fd.seed, j, uint32_t(i), PURPOSE_PROP, uint32_t(mm) * (N / per_block));
      R Fv[N];
#pragma unroll
      for (int n = 0; n < N; ++n) Fv[n] = fmaR(sw, z[n], F);
      l96_rk4_step_f<N, R>(x, [&](int n) { return Fv[n]; }, dt, h2, h3, h6);
    }
  }
}

// Lorenz '96 weight: sum over observed components (index order) of
// (y - x_n)^2 accumulated by fma in FP64, times cw = -0.5 / r.
template <int N, typename R>
__device__ __forceinline__ double l96_weight(const FilterDev& fd, const R (&x)[N],
                                             const double* ys, double cw) {
  const uint64_t mask = fd.obs_mask;
  double acc = 0.0;
  int k = 0;
#pragma unroll
  for (int n = 0; n < N; ++n) {
    if ((mask >> n) & 1ull) {
      const double d = ys[k] - to_double(x[n]);
      acc = fma(d, d, acc);
      ++k;
    }
  }
  return acc * cw;
}

// ---------------------------------------------------------------------------
// Group and filter combines (run by the last block to finish).
// ---------------------------------------------------------------------------
struct CombineScratch {
  BlockScratch b;
  double incl[TILE];
  double gM, gS, gQ;  // thread 0's group partials, for a one-group filter's combine
  double tg[MAX_CLUSTER_TILES], tbase[MAX_CLUSTER_TILES];  // warp path: the first tiles' g, base
  double G;           // one-group filter: the group scale the filter combine took
  int last;
};

// Combine the tile partials of group g: group max, tile scales g_t =
// exp(M_t - M_g), inclusive scan of S_t g_t (tile bases = exclusive prefix),
// group sum = scan total.  Returns true in every thread of the block that
// finished the filter's last group.  With WARP, a group of at most 32 tiles is
// combined by warp 0 alone, and the only group of a filter skips the group
// ticket (it is the last by construction); both give the same bits as the
// block path.
// The tile partials (M, S, Q) of a cluster's tiles, gathered in CTA 0's shared
// memory (the values propagate_tile also writes to tp); src = nullptr: read
// them from tp.
struct TileTriples {
  double M[MAX_CLUSTER_TILES], S[MAX_CLUSTER_TILES], Q[MAX_CLUSTER_TILES];
};

// store = false (the cluster path's CTAs other than the first, which combine
// the same partials for themselves): the global copies (tp, gp) are left to
// the CTA that stores them.
template <bool WARP, bool OWN>
__device__ bool combine_group(const FilterDev& fd, int g, CombineScratch& cs,
                              const TileTriples* src = nullptr, bool store = true) {
  const int tid = threadIdx.x;
  const int t0 = g * GROUP;
  const int ntg = min(GROUP, fd.ntiles - t0);
  double Mg = -INFINITY, Sg = 0.0, Qg = 0.0;  // thread 0's values are stored
  if (WARP && ntg <= 32) {
    // warp 0 alone (warp_max / warp_scan / warp_sum: the same bits)
    if (tid < 32) {
      double Mt = -INFINITY, St = 0.0, Qt = 0.0;
      if (tid < ntg) {
        if (src) {
          Mt = src->M[tid];
          St = src->S[tid];
          Qt = src->Q[tid];
        } else {
          Mt = ldcg(&fd.tp[t0 + tid].M);
          St = ldcg(&fd.tp[t0 + tid].S);
          Qt = ldcg(&fd.tp[t0 + tid].Q);
        }
      }
      Mg = warp_max(Mt);
      // exp(0) = 1 exactly: the maximal tile (and a one-tile group) skips the call
      const double gt = (Mt == -INFINITY) ? 0.0 : (Mt == Mg ? 1.0 : combine_exp<OWN>(Mt - Mg));
      const double incl = warp_scan(St * gt, &Sg);
      if (fd.mode == MODE_ADAPTIVE) Qg = warp_sum(Qt * (gt * gt));
      const double before = __shfl_up_sync(0xffffffffu, incl, 1);
      if (store && tid < ntg) {
        fd.tp[t0 + tid].g = gt;
        fd.tp[t0 + tid].base = tid == 0 ? 0.0 : before;
      }
      if (tid < MAX_CLUSTER_TILES) {  // warp 0's lanes keep their tile's g and base
        cs.tg[tid] = gt;
        cs.tbase[tid] = tid == 0 ? 0.0 : before;
      }
    }
  } else {
    double Mt = -INFINITY, St = 0.0, Qt = 0.0;
    if (tid < ntg) {
      Mt = ldcg(&fd.tp[t0 + tid].M);
      St = ldcg(&fd.tp[t0 + tid].S);
      Qt = ldcg(&fd.tp[t0 + tid].Q);
    }
    Mg = block_max(Mt, cs.b);
    const double gt = (Mt == -INFINITY) ? 0.0 : combine_exp<OWN>(Mt - Mg);
    const double incl = block_scan(St * gt, cs.b, &Sg);
    cs.incl[tid] = incl;
    if (fd.mode == MODE_ADAPTIVE) Qg = block_sum(Qt * (gt * gt), cs.b);
    __syncthreads();
    if (tid < ntg) {
      fd.tp[t0 + tid].g = gt;
      fd.tp[t0 + tid].base = tid == 0 ? 0.0 : cs.incl[tid - 1];
    }
  }
  if (tid == 0) {
    if (store) {
      GroupPart& gp = fd.gp[g];
      gp.M = Mg;
      gp.S = Sg;
      gp.Q = Qg;
      gp.ticket = 0u;
    }
    cs.gM = Mg;
    cs.gS = Sg;
    cs.gQ = Qg;
  }
  // the only group of a filter is its last: no ticket, and the filter
  // combine's warp 0 reads this group's partials back in thread 0
  if (WARP && fd.ngroups == 1) return true;
  if (tid == 0) {
    __threadfence();
    const unsigned old = atomicAdd(&fd.ctl->gticket, 1u);
    cs.last = (old == unsigned(fd.ngroups - 1));
  }
  __syncthreads();
  const bool last = cs.last != 0;
  if (last) __threadfence();
  return last;
}

// Combine the groups of the filter and take the step's decisions (with WARP,
// by warp 0 alone for at most 32 groups: the same bits).  sctl, when given, is
// a copy of the control block in shared memory (the cluster path's): the
// decisions are read from and taken in it, then the whole block is stored to
// fd.ctl at once (only with store; store = false also leaves gp alone).
// u_pre, when given, is the step's resampling uniform drawn ahead by another
// thread (the same value this function would draw).
template <bool WARP, bool OWN>
__device__ void combine_filter(const FilterDev& fd, int i, CombineScratch& cs,
                               Ctl* sctl = nullptr, bool store = true,
                               const double* u_pre = nullptr) {
  const int tid = threadIdx.x;
  const int ng = fd.ngroups;
  double M, S, Q = 0.0;
  if (WARP && ng == 1) {
    // one group: M = M_g, G = exp(0) = 1, S = S_g, Q = Q_g, B = 0 -- what the
    // reductions below give, without reading the partials back
    if (tid != 0) return;
    M = cs.gM;
    const double G = (M == -INFINITY) ? 0.0 : 1.0;
    S = cs.gS * G;
    if (fd.mode == MODE_ADAPTIVE) Q = cs.gQ * (G * G);
    if (store) {
      fd.gp[0].G = G;
      fd.gp[0].B = 0.0;
    }
    cs.G = G;
  } else if (WARP && ng <= 32) {
    // warp 0 alone (the same bits as the block reductions)
    if (tid >= 32) return;
    double Mg = -INFINITY, Sg = 0.0, Qg = 0.0;
    if (tid < ng) {
      Mg = ldcg(&fd.gp[tid].M);
      Sg = ldcg(&fd.gp[tid].S);
      Qg = ldcg(&fd.gp[tid].Q);
    }
    M = warp_max(Mg);
    const double G = (Mg == -INFINITY) ? 0.0 : combine_exp<OWN>(Mg - M);
    const double incl = warp_scan(Sg * G, &S);
    if (fd.mode == MODE_ADAPTIVE) Q = warp_sum(Qg * (G * G));
    const double before = __shfl_up_sync(0xffffffffu, incl, 1);
    if (tid < ng) {
      fd.gp[tid].G = G;
      fd.gp[tid].B = tid == 0 ? 0.0 : before;
    }
  } else {
    double Mg = -INFINITY, Sg = 0.0, Qg = 0.0;
    if (tid < ng) {
      Mg = ldcg(&fd.gp[tid].M);
      Sg = ldcg(&fd.gp[tid].S);
      Qg = ldcg(&fd.gp[tid].Q);
    }
    M = block_max(Mg, cs.b);
    const double G = (Mg == -INFINITY) ? 0.0 : combine_exp<OWN>(Mg - M);
    const double incl = block_scan(Sg * G, cs.b, &S);
    cs.incl[tid] = incl;
    if (fd.mode == MODE_ADAPTIVE) Q = block_sum(Qg * (G * G), cs.b);
    __syncthreads();
    if (tid < ng) {
      fd.gp[tid].G = G;
      fd.gp[tid].B = tid == 0 ? 0.0 : cs.incl[tid - 1];
    }
  }
  if (tid == 0) {
    Ctl* c = sctl ? sctl : fd.ctl;
    c->gticket = 0u;
    c->rs_step = i;
    if (!(M > -INFINITY) || M == INFINITY || !(S > 0.0)) {
      c->status = ST_DEGENERATE;
      c->ll = -INFINITY;
      c->rs_flag = 0;
      c->step = fd.T + 1;
    } else if (!(fd.obs_every == 1 || i % fd.obs_every == 0)) {
      // no observation at t_i: no likelihood term, no resampling, the
      // carried weights stay as they are (M = 0 makes the carry an identity)
      c->M = 0.0;
      c->S = S;
      c->rs_flag = 0;
      if (i < fd.T) c->anc_identity = 1;
      c->step = i + 1;
    } else {
      const double incr = ((M + combine_log<OWN>(S)) - c->L) + c->c_obs;
      c->ll = c->ll + incr;
      bool resample = false;
      if (i < fd.T) {
        if (fd.mode == MODE_ALWAYS) resample = true;
        else if (fd.mode == MODE_ADAPTIVE) resample = (S * S) / Q < fd.thr * double(fd.P);
      }
      c->M = M;
      c->S = S;
      if (resample) {
        c->u = u_pre ? *u_pre : resample_uniform(fd, i);
        c->ratio = double(fd.P) / S;
        c->rs_flag = 1;
        c->anc_identity = 0;
        c->lam_zero = 1;
        c->L = c->logP;
      } else {
        c->rs_flag = 0;
        if (i < fd.T) {
          c->anc_identity = 1;
          c->lam_zero = 0;
          c->L = combine_log<OWN>(S);
        }
      }
      c->step = i + 1;
    }
    if (sctl && store) *fd.ctl = *sctl;
  }
}

// ---------------------------------------------------------------------------
// Kernels
// ---------------------------------------------------------------------------
// Initial draw of tile t of a filter (Algorithm 2, initialise lines): x_n^j(t_0)
// = m0 + s0 z_n; tile 0 also resets the control block.
template <int KIND, int N, typename R>
__device__ __forceinline__ void init_tile(const FilterDev& fd, int t) {
  const int j = t * TILE + threadIdx.x;
  const int P = fd.P;
  const double m0 = wk_kind(KIND) ? fd.theta[5] : fd.theta[3];
  const double s0 = wk_kind(KIND) ? fd.theta[6] : fd.theta[4];
  if (j < P) {
    R z[N];
    normals<N>(z, fd.seed, uint32_t(j), 0u, PURPOSE_INIT);
    R* x0 = static_cast<R*>(fd.x[0]);
#pragma unroll
    for (int n = 0; n < N; ++n)
      x0[int64_t(n) * P + j] = fmaR(from_double<R>(s0), z[n], from_double<R>(m0));
    if (fd.hist) fd.anc[j] = j;
  }
  if (threadIdx.x == 0 && (t % GROUP) == 0) fd.gp[t / GROUP].ticket = 0u;
  if (threadIdx.x == 0) fd.tp[t].ticket = 0u;
  if (threadIdx.x == 0 && t == 0) {
    Ctl* c = fd.ctl;
    const double r = wk_kind(KIND) ? fd.theta[4] : fd.theta[2];
    c->step = 1;
    c->rs_step = 0;
    c->rs_flag = 0;
    c->anc_identity = 1;
    c->lam_zero = 1;
    c->status = ST_OK;
    c->gticket = 0u;
    c->rticket = 0u;
    c->ll = 0.0;
    c->logP = log(double(P));
    c->L = c->logP;
    c->c_obs = -0.5 * double(fd.Ny) * log(2.0 * 3.141592653589793 * r);
    c->cw = -0.5 / r;
    c->M = 0.0;
    c->S = 0.0;
    c->u = 0.0;
    c->ratio = 0.0;
    if (l96_kind(KIND)) l96_constants32(fd, c->lf);
  }
}

template <int KIND, int N, typename R>
__global__ void __launch_bounds__(TILE) k_init(const FilterDev* __restrict__ fds,
                                               const int2* __restrict__ tmap) {
  const int2 ft = tmap[blockIdx.x];
  init_tile<KIND, N, R>(fds[ft.x], ft.y);
}

// Blocks per SM the propagate kernel is compiled for (registers per thread =
// 65536 / (256 x blocks)).  The small states are bound by FP64 latency, so
// more resident warps pay, up to a few spilled words (each step measured
// faster than the one before it): FP32 windkessel 8 (32 registers, 28 bytes
// spilled), FP64 windkessel 4 (64); Lorenz '96 in FP32: N = 4 and N = 8 5
// (48; N = 8 spills 32 bytes), N = 12 3 (85), larger N 2 (the N = 40 state
// needs its 128 registers); in FP64 2 up to N = 12, else 1.
template <int KIND, int N, typename R>
struct PropagateOccupancy {
  static constexpr int value = (wk_kind(KIND) && sizeof(R) == 4) ? 8
                               : wk_kind(KIND)                    ? 4
                               : (sizeof(R) == 4 && N <= 4)      ? 5
                               : (sizeof(R) == 4 && N <= 8)      ? 5
                               : (sizeof(R) == 4 && N <= 12)     ? 3
                               : (sizeof(R) == 4 || N <= 12)     ? 2
                                                                 : 1;
};

// Address of the same shared-memory object in CTA `rank` of the cluster
// (distributed shared memory: a generic pointer the other CTA can store to).
template <typename T>
__device__ __forceinline__ T* cluster_peer(T* local, unsigned rank) {
  unsigned long long out;
  asm volatile("mapa.u64 %0, %1, %2;" : "=l"(out) : "l"(reinterpret_cast<unsigned long long>(local)),
               "r"(rank));
  return reinterpret_cast<T*>(out);
}

// Step i of tile t (Algorithm 2, propagate and weight lines), propagate_tile
// below: gather the ancestors' states, propagate, store, weight with y(t_i) in
// FP64 (skipped at a step without an observation), then the tile partials:
// max, inclusive prefix of exp(ell - M_t) (ctil) and its total; thread 0
// writes them to tp[t].  a_spec is the ancestor row's entry when there is no
// history (loaded early).  tri (the cluster path): this CTA's TileTriples;
// thread 0 also stores the tile's partials into that object in each of the
// cluster's first ncopies CTAs.
// Its two parts, which the sub-tile launch (k_propagate_sub) also calls:
// propagate_ell (every thread of the block calls it; particle j, when valid,
// is gathered, propagated, stored and weighted: its log-weight is returned,
// -inf for an invalid slot) and tile_epilogue (the tile's reductions over the
// 256 log-weights of tile t, thread k holding particle j = 256 t + k).
template <int KIND, int N, typename R>
__device__ __forceinline__ double propagate_ell(const FilterDev& fd, int i, int j, bool valid,
                                                int anc_identity, int lam_zero, double cw,
                                                int a_spec, double* ys,
                                                const float* lf = nullptr) {
  const int P = fd.P;
  const int tid = threadIdx.x;
  if (tid < fd.Ny) ys[tid] = fd.y[int64_t(i - 1) * fd.Ny + tid];  // read after the barrier below

  __shared__ R kc[3];  // per-filter constants of the exact windkessel
  if constexpr (KIND == KIND_WKX) {
    if (tid == 0) wkx_constants<R>(fd, kc);
    __syncthreads();
  }
  // Euler windkessel: F(t_k)/C of the step's substeps, one division each, and
  // the filter's sqrt(q), RC, C and dt in R, converted by one thread per block
  // (conversions from FP64 run on the FP64 unit, which bounds this kernel)
  __shared__ R fcs[KIND == KIND_WK ? TILE : 1];
  __shared__ R wkc[4];
  const R* fc = nullptr;
  if constexpr (KIND == KIND_WK) {
    if (tid == TILE - 2) {
      wkc[0] = sqrt(from_double<R>(fd.theta[3]));
      wkc[1] = from_double<R>(fd.theta[0]) * from_double<R>(fd.theta[1]);
      wkc[2] = from_double<R>(fd.theta[1]);
      wkc[3] = from_double<R>(fd.dt);
    }
    if (fd.s <= TILE) {
      if (tid < fd.s)
        fcs[tid] = from_double<R>(fd.flow[int64_t(i - 1) * fd.s + tid]) /
                   from_double<R>(fd.theta[1]);
      fc = fcs;
    }
    __syncthreads();
  }
  R x[N];
  if (valid) {
    int a = anc_identity ? j : (fd.hist ? fd.anc[int64_t(i - 1) * P + j] : a_spec);
    if constexpr (PF_CHECKED) {
      if (a < 0 || a >= P) {
        check_failed(CHK_ANCESTOR);
        a = j;
      }
    }
    const R* xin = static_cast<const R*>(fd.x[(i - 1) & 1]);
    R* xout = static_cast<R*>(fd.x[i & 1]);
#pragma unroll
    for (int n = 0; n < N; ++n) x[n] = xin[int64_t(n) * P + a];
    if constexpr (KIND == KIND_WK) wk_propagate<R>(fd, uint32_t(j), i, x[0], fc, wkc);
    else if constexpr (KIND == KIND_WKX) wkx_propagate<R>(fd, uint32_t(j), i, x[0], kc);
    else if constexpr (KIND == KIND_L96W) l96w_propagate<N, R>(fd, uint32_t(j), i, x);
    else l96_propagate<N, R>(fd, uint32_t(j), i, x, lf);
    if constexpr (PF_CHECKED) {
      bool bad = false;
#pragma unroll
      for (int n = 0; n < N; ++n) bad |= !isfinite(x[n]);
      if (bad) check_failed(CHK_STATE);
    }
#pragma unroll
    for (int n = 0; n < N; ++n) xout[int64_t(n) * P + j] = x[n];
  }
  __syncthreads();  // observation row staged
  double ell = -INFINITY;
  const bool observed = fd.obs_every == 1 || i % fd.obs_every == 0;
  if (valid) {
    double lw = 0.0;  // a step without an observation carries the weights
    if (observed) {
      if constexpr (wk_kind(KIND)) lw = wk_weight<R>(fd, i, x[0], ys[0], cw);
      else lw = l96_weight<N, R>(fd, x, ys, cw);
    }
    double e = lam_zero ? lw : fd.lam[j] + lw;
    // NaN -> -inf, tested on the bits (an FP64 compare is FP64-unit work)
    if ((static_cast<unsigned long long>(__double_as_longlong(e)) & 0x7fffffffffffffffull) >
        0x7ff0000000000000ull)
      e = -INFINITY;
    ell = e;
    if (fd.mode != MODE_ALWAYS) fd.ell[j] = e;
  }
  return ell;
}

template <bool FIXED>
__device__ __forceinline__ void tile_epilogue(const FilterDev& fd, int t, int j, double ell,
                                              CombineScratch& cs, TileTriples* tri = nullptr,
                                              int ncopies = 0) {
  const int P = fd.P;
  const int tid = threadIdx.x;
  // tile partials: max, inclusive prefix of exp(ell - M_t) (FIXED: exact sums
  // of the weights in 2^-55 fixed point, each rounded once to a double), total
  const double Mt = block_max(ell, cs.b);
  const double w = (static_cast<unsigned long long>(__double_as_longlong(Mt)) ==
                    0xfff0000000000000ull)  // Mt == -inf, on the bits
                       ? 0.0
                       : exp_weight(ell - Mt);
  double c, St;
  if constexpr (FIXED) {
    unsigned long long Ft;
    c = fixed_double(block_scan_fixed(weight_fixed(w), cs.b, &Ft));
    St = fixed_double(Ft);
  } else {
    c = block_scan(w, cs.b, &St);
  }
  if constexpr (PF_CHECKED) {
    // FIXED: the prefixes are non-decreasing by construction (an exact integer
    // scan, rounded monotonically).  Otherwise neighbouring prefixes come from
    // different addition trees and may differ by rounding (at most about ten
    // ulp: five levels of sums of non-negative terms).  A weight above 1 or a
    // larger decrease is a violation.
    const double before = __shfl_up_sync(0xffffffffu, c, 1);
    const double floor_ = FIXED ? before : before * (1.0 - 0x1p-49);
    if (j < P && (!(c >= 0.0) || !(w <= 1.0) || ((tid & 31) > 0 && c < floor_)))
      check_failed(CHK_PREFIX);
  }
  if (j < P) fd.ctil[j] = c;
  double Qt = 0.0;
  if (fd.mode == MODE_ADAPTIVE) Qt = block_sum(w * w, cs.b);
  if (tid == 0) {
    TilePart& tp = fd.tp[t];
    tp.M = Mt;
    tp.S = St;
    tp.Q = Qt;
    for (int r = 0; r < ncopies; ++r) {  // the cluster path: into every CTA's shared memory
      TileTriples* dst = cluster_peer(tri, unsigned(r));
      dst->M[t] = Mt;
      dst->S[t] = St;
      dst->Q[t] = Qt;
    }
  }
}

template <int KIND, int N, typename R>
__device__ __forceinline__ void propagate_tile(const FilterDev& fd, int t, int i, int anc_identity,
                                               int lam_zero, double cw, int a_spec, double* ys,
                                               CombineScratch& cs, TileTriples* tri = nullptr,
                                               int ncopies = 0, const float* lf = nullptr) {
  const int j = t * TILE + int(threadIdx.x);
  const double ell = propagate_ell<KIND, N, R>(fd, i, j, j < fd.P, anc_identity, lam_zero, cw,
                                               a_spec, ys, lf);
  tile_epilogue<FixedPrefix<KIND, N>::value>(fd, t, j, ell, cs, tri, ncopies);
}

// The step kernels are launched with programmatic stream serialization: the
// next one in the stream may be launched while this one drains, and waits
// here, before its first read, until the previous grid has completed and its
// writes are visible (a hardware wait; a no-op without the launch attribute).
__device__ __forceinline__ void wait_prior_grid() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
}

template <int KIND, int N, typename R>
__global__ void __launch_bounds__(TILE, (PropagateOccupancy<KIND, N, R>::value)) k_propagate(const FilterDev* __restrict__ fds,
                                                    const int2* __restrict__ tmap) {
  __shared__ CombineScratch cs;
  __shared__ double ys[64];
  wait_prior_grid();
  const int2 ft = tmap[blockIdx.x];
  const FilterDev& fd = fds[ft.x];
  Ctl* ctl = fd.ctl;
  const int P = fd.P;
  const int t = ft.y;
  const int tid = threadIdx.x;
  const int j = t * TILE + tid;
  const bool valid = j < P;
  // issued before the control block is read (without a history the ancestor
  // row does not depend on the step), so the two loads overlap
  const int a_spec = (valid && !fd.hist) ? fd.anc[j] : j;
  // one thread reads the control block (written by the previous launch) and
  // shares it: every thread reading it would queue on one L2 line
  __shared__ int s_step, s_ok, s_anc_identity, s_lam_zero;
  __shared__ double s_cw;
  // the FP32 small-state Lorenz '96 constants of the run (see l96_constants32)
  constexpr bool LF = KIND == KIND_L96 && sizeof(R) == 4 && N <= 12;
  __shared__ float s_lf[LF ? 6 : 1];
  if (tid == 0) {
    s_step = ldcg(&ctl->step);
    s_ok = ldcg(&ctl->status) == ST_OK;
    s_anc_identity = ldcg(&ctl->anc_identity);
    s_lam_zero = ldcg(&ctl->lam_zero);
    s_cw = ldcg(&ctl->cw);
    if constexpr (LF) {
#pragma unroll
      for (int k = 0; k < 6; ++k) s_lf[k] = ldcg(&ctl->lf[k]);
    }
  }
  __syncthreads();
  const int i = s_step;
  if (i > fd.T || !s_ok) return;
  propagate_tile<KIND, N, R>(fd, t, i, s_anc_identity, s_lam_zero, s_cw, a_spec, ys, cs, nullptr,
                             0, LF ? s_lf : nullptr);
  if (tid == 0) {
    __threadfence();
    const int g = t / GROUP;
    const int ntg = min(GROUP, fd.ntiles - g * GROUP);
    const unsigned old = atomicAdd(&fd.gp[g].ticket, 1u);
    cs.last = (old == unsigned(ntg - 1));
  }
  __syncthreads();
  if (!cs.last) return;
  __threadfence();
  // the large states keep the block reductions only: the extra code of the
  // warp paths measurably slows their register-bound main loop (same bits)
  constexpr bool WARP = !(l96_kind(KIND) && N >= 16);
  constexpr bool OWN = OwnCombineMath<KIND, N>::value;
  if (combine_group<WARP, OWN>(fd, t / GROUP, cs)) combine_filter<WARP, OWN>(fd, i, cs);
}

// The same step with each tile propagated by SUB blocks, block (t, h) taking
// particles [256 t + h 256/SUB, 256 t + (h+1) 256/SUB) with its first 256/SUB
// threads (the others only join the block's barriers): for a small filter of
// FP64 state, whose tiles would leave most SMs idle while each runs its FP64
// work (B300: 1/64 of the FP32 rate), the work of a tile spreads over SUB
// SMs.  Each block parks its particles' log-weights in ctil; the last of the
// tile's SUB blocks (tp[t].ticket) reads the tile's 256 back and runs
// tile_epilogue and the combines exactly as k_propagate does, so every
// result is bit-identical to k_propagate's.
template <int KIND, int N, typename R, int SUB>
__global__ void __launch_bounds__(TILE, (PropagateOccupancy<KIND, N, R>::value))
    k_propagate_sub(const FilterDev* __restrict__ fds, const int2* __restrict__ tmap) {
  static_assert(SUB == 2 || SUB == 4, "two or four blocks per tile");
  constexpr int PART = TILE / SUB;
  __shared__ CombineScratch cs;
  __shared__ double ys[64];
  wait_prior_grid();
  const int2 ft = tmap[blockIdx.x / SUB];
  const int h = int(blockIdx.x % SUB);
  const FilterDev& fd = fds[ft.x];
  Ctl* ctl = fd.ctl;
  const int P = fd.P;
  const int t = ft.y;
  const int tid = threadIdx.x;
  const int j = t * TILE + h * PART + tid;
  const bool valid = tid < PART && j < P;
  const int a_spec = (valid && !fd.hist) ? fd.anc[j] : j;
  __shared__ int s_step, s_ok, s_anc_identity, s_lam_zero;
  __shared__ double s_cw;
  if (tid == 0) {
    s_step = ldcg(&ctl->step);
    s_ok = ldcg(&ctl->status) == ST_OK;
    s_anc_identity = ldcg(&ctl->anc_identity);
    s_lam_zero = ldcg(&ctl->lam_zero);
    s_cw = ldcg(&ctl->cw);
  }
  __syncthreads();
  const int i = s_step;
  if (i > fd.T || !s_ok) return;
  const double ell =
      propagate_ell<KIND, N, R>(fd, i, j, valid, s_anc_identity, s_lam_zero, s_cw, a_spec, ys);
  if (valid) fd.ctil[j] = ell;  // parked for the tile's epilogue
  __syncthreads();              // the part's states and log-weights, before its ticket
  if (tid == 0) {
    __threadfence();
    cs.last = atomicAdd(&fd.tp[t].ticket, 1u) == unsigned(SUB - 1);
  }
  __syncthreads();
  if (!cs.last) return;
  __threadfence();
  if (tid == 0) fd.tp[t].ticket = 0u;  // for the next step (ordered by the launch boundary)
  const int jt = t * TILE + tid;
  tile_epilogue<FixedPrefix<KIND, N>::value>(fd, t, jt, jt < P ? ldcg(&fd.ctil[jt]) : -INFINITY,
                                              cs);
  if (tid == 0) {
    __threadfence();
    const int g = t / GROUP;
    const int ntg = min(GROUP, fd.ntiles - g * GROUP);
    const unsigned old = atomicAdd(&fd.gp[g].ticket, 1u);
    cs.last = (old == unsigned(ntg - 1));
  }
  __syncthreads();
  if (!cs.last) return;
  __threadfence();
  constexpr bool WARP = !(l96_kind(KIND) && N >= 16);
  constexpr bool OWN = OwnCombineMath<KIND, N>::value;
  if (combine_group<WARP, OWN>(fd, t / GROUP, cs)) combine_filter<WARP, OWN>(fd, i, cs);
}

// Number of systematic targets j in [0, P) below cumulative weight b: target
// j sits at (j + u) S / P, compared in the scaled form j < b (P / S) - u, so
// the count is ceil(b ratio - u) clamped to [0, P].
__device__ __forceinline__ int targets_below(double b, double ratio, double u, int P) {
  const double e = b * ratio - u;
  if (!(e > 0.0)) return 0;
  if (e >= double(P)) return P;
  return __double2int_ru(e);
}

// The same count for a particle of a tile whose cumulative weights are
// C_k = base + scale * prefix_k, evaluated as ceil(fma(scale', prefix_k, e0))
// with scale' = scale ratio and e0 = base ratio - u prepared once per tile
// (one FP64 fma per particle; the conversion saturates, and the caller clamps
// the count to the tile's own target range).
__device__ __forceinline__ int ceil_count(double e) {
  // ceil(e) read off the bits with integer operations (B300's FP64 unit, at
  // 1/64 of the FP32 rate, would spend several cycles on the conversion):
  // 0 for e <= 0, the exact ceiling for 0 < e < 2^30, a large count above
  // (callers clamp the count to the tile's range).
  const long long b = __double_as_longlong(e);
  if (b <= 0) return 0;  // +0, negative values (and -NaN)
  const int ex = int(b >> 52) - 1023;
  if (ex < 0) return 1;  // 0 < e < 1
  if (ex >= 30) return 0x7fffffff;
  const long long m = (b & 0x000fffffffffffffLL) | 0x0010000000000000LL;
  const int sh = 52 - ex;
  const long long ip = m >> sh;
  return int(ip) + ((m & ((1LL << sh) - 1)) != 0 ? 1 : 0);
}

__device__ __forceinline__ int tile_targets_below(double scale_r, double prefix, double e0) {
  return ceil_count(fma(scale_r, prefix, e0));
}

// Stratified count: targets j + u_j (u_j from Philox block (j, i, RESAMPLE, 1))
// below the scaled cumulative weight e: every j < floor(e), plus j = floor(e)
// when e - floor(e) > u_j (exact, since e - floor(e) is exact).
// Both parts are read off the bits with integer operations, so the test
// frac(e) > u_j (u_j = v 2^-53, v the 53-bit integer of the uniform) is exact:
// for e >= 1, floor(e) is the 53-bit mantissa m shifted right by 52 - ex and
// frac(e) 2^53 the remaining bits shifted left by ex + 1; for e < 1,
// e 2^53 = m 2^(ex+1) is compared through its integer part and whether
// anything was shifted out.
__device__ __forceinline__ int strat_below(double e, uint64_t seed, int i, int P) {
  const long long b = __double_as_longlong(e);
  if (b <= 0) return 0;  // e <= 0
  if (e >= double(P)) return P;
  const int ex = int(b >> 52) - 1023;
  const unsigned long long m = (b & 0x000fffffffffffffLL) | 0x0010000000000000LL;
  unsigned long long q;  // integer part of frac(e) 2^53
  bool rem = false;      // frac(e) 2^53 is not an integer
  int f = 0;
  if (ex >= 0) {
    const int sh = 52 - ex;
    f = int(m >> sh);
    q = (m & ((1ull << sh) - 1ull)) << (ex + 1);
  } else {
    const int k = -(ex + 1);
    q = k < 53 ? m >> k : 0ull;
    rem = k < 53 ? (m & ((1ull << k) - 1ull)) != 0ull : true;
  }
  const uint4 w = rng_block(seed, uint32_t(f), uint32_t(i), PURPOSE_RESAMPLE, 1u);
  const unsigned long long v = ((static_cast<unsigned long long>(w.y) << 32) | w.x) >> 11;
  return f + ((q > v || (q == v && rem)) ? 1 : 0);
}

// Multinomial count: the number of targets (mn_t, scaled and sorted) below e,
// searched in [lo, hi].
__device__ __forceinline__ int mn_below(const FilterDev& fd, double e, int lo, int hi) {
  while (lo < hi) {
    const int mid = lo + (hi - lo) / 2;
    if (ldcg(&fd.mn_t[mid]) < e) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// Resampling of one tile.  Its particles k have cumulative weights
// C_k = base + scale * prefix_k; the tile owns the targets [lo, hi) between
// its base and the next tile's base (both counts computed from the same
// values in the two tiles), and particle k takes the targets [n_{k-1}, n_k)
// with n_k = the count of targets below C_k, clamped to [lo, hi] (the last
// particle takes the rest).  Counts: systematic ceil(C (P/S) - u); stratified
// and multinomial as strat_below / mn_below on C (P/S).  Only the counts use
// FP64 (one fma per particle; ceilings and floors are taken on the bits).
//
// Barriers: two per chunk of tiles (after their ranges and scaled bases are
// prepared, after the counts), one vote per chunk for very long offspring
// ranges (written by the whole block after it), one at the end of the chunk.  A particle's predecessor
// count comes from the neighbouring lane (lane 0's from the running maximum
// of the earlier warps' last counts, through shared memory); ranges up to
// SHORT_RANGE are written by the particle's thread, up
// to BLOCK_RANGE by its warp, longer ones by the whole block, so a tile that
// owns most of the targets still writes them with coalesced stores.
constexpr int SHORT_RANGE = 16;
constexpr int BLOCK_RANGE = 2048;
constexpr int RESAMPLE_BLOCKS_PER_SM = 8;

// Tile t's cumulative weights are C_k = base + scale * prefix_k: which = 0
// gives this tile's base and scale, which = 1 the next tile's base (S after the
// last tile), from the group and tile partials of the filter combine.
__device__ __forceinline__ void tile_base(const FilterDev& fd, int t, int which, double S,
                                          double* base, double* scale) {
  if (which == 0) {
    const int g = t / GROUP;
    const double gG = fd.gp[g].G;
    *base = fma(gG, fd.tp[t].base, fd.gp[g].B);
    *scale = gG * fd.tp[t].g;
  } else if (t + 1 < fd.ntiles) {
    const int g1 = (t + 1) / GROUP;
    *base = fma(fd.gp[g1].G, fd.tp[t + 1].base, fd.gp[g1].B);
  } else {
    *base = S;
  }
}

// The count of targets below a tile end, per scheme.
__device__ __forceinline__ int range_count(const FilterDev& fd, int rs, double base, double ratio,
                                           double u, int i) {
  if (rs == RS_SYSTEMATIC) return targets_below(base, ratio, u, fd.P);
  if (rs == RS_STRATIFIED) return strat_below(base * ratio, fd.seed, i, fd.P);
  return mn_below(fd, base * ratio, 0, fd.P);
}

// The offspring ranges longer than BLOCK_RANGE of one tile, written by the
// whole block with coalesced stores.
__device__ __forceinline__ void write_long_ranges(int32_t* aout, int nl, const int3* longr) {
  for (int r = 0; r < nl; ++r) {
    const int3 rg = longr[r];
    for (int jj = rg.x + int(threadIdx.x); jj < rg.y; jj += TILE) aout[jj] = rg.z;
  }
}

// The count of targets below a particle's scaled cumulative weight (in-tile
// prefix c), by scheme, clamped to its tile's target range [lo, hi].
__device__ __forceinline__ int particle_count(const FilterDev& fd, int i, int rs, int lo, int hi,
                                              double e0, double scale_r, double c) {
  int n;
  if (rs == RS_SYSTEMATIC) n = tile_targets_below(scale_r, c, e0);
  else if (rs == RS_STRATIFIED) n = strat_below(fma(scale_r, c, e0), fd.seed, i, fd.P);
  else n = mn_below(fd, fma(scale_r, c, e0), lo, hi);
  return min(max(n, lo), hi);
}

// Particle j of tile t takes the targets [prev, n) as ancestor: written by its
// thread or its warp; a range longer than BLOCK_RANGE is only listed in
// longr (returns true), for the whole block to write after a block vote.
// Every thread of the warp calls it; no block barrier.
__device__ __forceinline__ bool write_offspring_local(const FilterDev& fd, int t, int i, int prev,
                                                      int n, bool valid, int* nlong,
                                                      int3* longr) {
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int j0 = t * TILE;
  const int j = j0 + tid;
  if (PF_CHECKED && valid && (n < prev || prev < 0 || n > fd.P)) check_failed(CHK_RANGE);
  const int len = valid ? n - prev : 0;
  int32_t* aout = fd.anc + (fd.hist ? int64_t(i) * fd.P : 0);
  if (len > 0 && len <= SHORT_RANGE)
    for (int jj = prev; jj < n; ++jj) aout[jj] = j;
  unsigned wl = __ballot_sync(0xffffffffu, len > SHORT_RANGE && len <= BLOCK_RANGE);
  while (wl) {
    const int src = __ffs(wl) - 1;
    wl &= wl - 1;
    const int a = __shfl_sync(0xffffffffu, prev, src);
    const int b = __shfl_sync(0xffffffffu, n, src);
    const int who = j0 + (tid & ~31) + src;
    for (int jj = a + lane; jj < b; jj += 32) aout[jj] = who;
  }
  if (len > BLOCK_RANGE) longr[atomicAdd(nlong, 1)] = make_int3(prev, n, j);
  return len > BLOCK_RANGE;
}

// write_offspring_local, then the tile's long ranges written by the whole
// block after a block vote.  Every thread of the block calls it (one barrier).
__device__ __forceinline__ void write_offspring(const FilterDev& fd, int t, int i, int prev, int n,
                                               bool valid, int* nlong, int3* longr) {
  const bool lng = write_offspring_local(fd, t, i, prev, n, valid, nlong, longr);
  if (__syncthreads_or(lng)) write_long_ranges(fd.anc + (fd.hist ? int64_t(i) * fd.P : 0), *nlong,
                                               longr);
}

// The running maximum of a count over the lanes of a warp.  The canonical
// in-tile scans are monotone only up to rounding (neighbouring prefixes come
// from different addition trees), so a count could in principle dip below
// its predecessor's when a target falls inside that ulp; taking the running
// maximum makes the offspring ranges disjoint and ordered by construction
// (and changes nothing otherwise).
__device__ __forceinline__ int warp_running_max(int n) {
  const int lane = threadIdx.x & 31;
  // nearly always the counts are monotone already: one shuffle and a vote
  const int up = __shfl_up_sync(0xffffffffu, n, 1);
  if (!__any_sync(0xffffffffu, lane > 0 && n < up)) return n;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, n, o);
    if (lane >= o) n = max(n, v);
  }
  return n;
}

// The particles of tile t take their targets [n_{k-1}, n_k): counts from the
// scaled cumulative weights (ct = this particle's in-tile prefix), made
// monotone over the tile (warp_running_max, then each warp's last count
// through shared memory); nlast: WARPS ints of shared scratch.
__device__ __forceinline__ void resample_particles(const FilterDev& fd, int t, int i, int rs,
                                                   int lo, int hi, double e0, double scale_r,
                                                   double ct, int* nlast, int* nlong,
                                                   int3* longr) {
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int w = tid >> 5;
  const int nvalid = min(TILE, fd.P - t * TILE);
  const bool valid = tid < nvalid;
  int n = (valid && tid != nvalid - 1) ? particle_count(fd, i, rs, lo, hi, e0, scale_r, ct) : hi;
  n = warp_running_max(n);
  if (lane == 31) nlast[w] = n;
  __syncthreads();
  int run = lo;
  for (int q = 0; q < w; ++q) run = max(run, nlast[q]);
  n = max(n, run);
  int prev = __shfl_up_sync(0xffffffffu, n, 1);
  if (lane == 0) prev = run;
  write_offspring(fd, t, i, prev, n, valid, nlong, longr);
}

// No resampling after step i: carry the log-weights (lam = ell - M) and, with
// a history, write the identity ancestor row.
__device__ __forceinline__ void carry_tile(const FilterDev& fd, int t, int i, double M) {
  const int j = t * TILE + threadIdx.x;
  if (j < fd.P) {
    if (fd.mode != MODE_ALWAYS) fd.lam[j] = fd.ell[j] - M;
    if (fd.hist) fd.anc[int64_t(i) * fd.P + j] = j;
  }
}

// A block takes the tiles q, q + G, q + 2G, ... of the tile map (G = the grid
// size, a multiple of the SM count) in chunks of up to RS_CHUNK tiles.  For a
// chunk, every thread first issues the loads of its particle's in-tile prefix
// in each tile, and lanes 2m and 2m + 1 of warp 0 read tile m's control block
// and compute the counts at its two ends (tile_base, range_count), so the
// dependent loads and FP64 operations of all the chunk's tiles overlap; then
// every particle's count in every tile of the chunk is taken, and each warp's
// last count passes through shared memory to the next warp's lane 0 (its
// predecessor), so no lane recomputes a count; then the tiles' offspring are
// written (or the tiles carried) one after the other (RS_CHUNK: pf_dev.cuh).

// Shared scratch of one chunk of resampled tiles.
struct RsChunk {
  int2 ft[RS_CHUNK];
  int i[RS_CHUNK], go[RS_CHUNK], flag[RS_CHUNK], lo[RS_CHUNK], hi[RS_CHUNK];
  int nlong[RS_CHUNK];
  double M[RS_CHUNK], e0[RS_CHUNK], sr[RS_CHUNK];
  int nlast[RS_CHUNK][WARPS];
  int3 longr[RS_CHUNK][TILE];  // each tile's offspring ranges longer than BLOCK_RANGE
};

// The chunk of the nq <= RS_CHUNK tiles tile_of(0..nq-1) (filter, tile),
// resampled or carried as described above.  The tiles' ranges longer than
// BLOCK_RANGE are listed while their short and warp-length ranges are
// written, then written by the whole block after one vote for the chunk.
// Every thread of the block calls it; it ends with a block barrier.
template <typename TileOf>
__device__ __forceinline__ void resample_chunk(const FilterDev* __restrict__ fds, TileOf tile_of,
                                               int nq, RsChunk& c) {
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int w = tid >> 5;
  double ct[RS_CHUNK];
#pragma unroll
  for (int m = 0; m < RS_CHUNK; ++m) {
    ct[m] = 0.0;
    if (m < nq) {
      const int2 ft = tile_of(m);
      const FilterDev& fd = fds[ft.x];
      const int j = ft.y * TILE + tid;
      if (j < fd.P) ct[m] = fd.ctil[j];
    }
  }
  if (tid < RS_CHUNK) c.nlong[tid] = 0;
  if (tid < 2 * nq) {
    const int m = tid >> 1, which = tid & 1;
    const int2 ft = tile_of(m);
    const FilterDev& fd = fds[ft.x];
    const Ctl* ctl = fd.ctl;
    const int rs = fd.resampler;
    const int i = ldcg(&ctl->rs_step);
    const int go = ldcg(&ctl->status) == ST_OK && i >= 1 && i < fd.T && ldcg(&ctl->step) == i + 1;
    const int flag = ldcg(&ctl->rs_flag);
    const double u = rs == RS_SYSTEMATIC ? ldcg(&ctl->u) : 0.0;
    const double ratio = ldcg(&ctl->ratio);
    double base = 0.0, scale = 0.0;
    tile_base(fd, ft.y, which, ldcg(&ctl->S), &base, &scale);
    const int n0 = (go && flag) ? range_count(fd, rs, base, ratio, u, i) : 0;
    if (which == 0) {
      c.ft[m] = ft;
      c.i[m] = i;
      c.go[m] = go;
      c.flag[m] = flag;
      c.M[m] = ldcg(&ctl->M);
      c.e0[m] = base * ratio - u;
      c.sr[m] = scale * ratio;
      c.lo[m] = n0;
    } else {
      c.hi[m] = n0;
    }
  }
  __syncthreads();
  // every particle's count in every tile of the chunk; each warp's last one
  // goes through shared memory to the next warp's lane 0
  int nn[RS_CHUNK];
#pragma unroll
  for (int m = 0; m < RS_CHUNK; ++m) {
    nn[m] = 0;
    if (m < nq && c.go[m] && c.flag[m]) {
      const int2 ft = c.ft[m];
      const FilterDev& fd = fds[ft.x];
      const int nvalid = min(TILE, fd.P - ft.y * TILE);
      nn[m] = (tid < nvalid && tid != nvalid - 1)
                  ? particle_count(fd, c.i[m], fd.resampler, c.lo[m], c.hi[m], c.e0[m], c.sr[m],
                                   ct[m])
                  : c.hi[m];
      nn[m] = warp_running_max(nn[m]);
      if (lane == 31) c.nlast[m][w] = nn[m];
    }
  }
  __syncthreads();
  bool lng = false;
#pragma unroll
  for (int m = 0; m < RS_CHUNK; ++m) {
    if (m < nq) {
      const int2 ft = c.ft[m];
      const FilterDev& fd = fds[ft.x];
      if (c.go[m] && c.flag[m]) {  // uniform over the block
        // the counts of the warps before this one bound this warp's below
        int run = c.lo[m];
        for (int q = 0; q < w; ++q) run = max(run, c.nlast[m][q]);
        nn[m] = max(nn[m], run);
        int prev = __shfl_up_sync(0xffffffffu, nn[m], 1);
        if (lane == 0) prev = run;
        const bool valid = tid < min(TILE, fd.P - ft.y * TILE);
        lng |= write_offspring_local(fd, ft.y, c.i[m], prev, nn[m], valid, &c.nlong[m],
                                     c.longr[m]);
      } else if (c.go[m]) {
        carry_tile(fd, ft.y, c.i[m], c.M[m]);
      }
    }
  }
  if (__syncthreads_or(lng)) {
#pragma unroll
    for (int m = 0; m < RS_CHUNK; ++m) {
      if (m < nq && c.nlong[m] > 0) {
        const FilterDev& fd = fds[c.ft[m].x];
        write_long_ranges(fd.anc + (fd.hist ? int64_t(c.i[m]) * fd.P : 0), c.nlong[m],
                          c.longr[m]);
      }
    }
  }
  __syncthreads();  // the chunk's shared values are rewritten by the next chunk
}

__global__ void __launch_bounds__(TILE, RESAMPLE_BLOCKS_PER_SM)
    k_resample(const FilterDev* __restrict__ fds, const int2* __restrict__ tmap, int ntiles) {
  __shared__ RsChunk c;
  const int G = gridDim.x;
  wait_prior_grid();
  for (int q0 = blockIdx.x; q0 < ntiles; q0 += RS_CHUNK * G) {
    const int nq = min(RS_CHUNK, (ntiles - q0 + G - 1) / G);  // q0 + m G < ntiles for m < nq
    resample_chunk(fds, [&](int m) { return tmap[q0 + m * G]; }, nq, c);
  }
}

// ---------------------------------------------------------------------------
// One thread-block cluster per small filter: the batched form's persistent path
// ---------------------------------------------------------------------------
// All the CTAs of a cluster wait here, with release / acquire semantics at
// cluster scope (every CTA of a cluster arrives the same number of times).
__device__ __forceinline__ void cluster_sync() {
  __threadfence();
  asm volatile("barrier.cluster.arrive.release.aligned;\n"
               "barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Filter list[blockIdx.x / CS] runs whole on a cluster of CS CTAs, CTA r
// owning tile r (CTAs past the filter's tiles take part in the barriers and
// the combine only): its initial draw, then per step its tiles propagated in
// parallel (propagate_tile), the group and the filter combined (combine_group,
// combine_filter), and its tiles resampled in parallel (resample_particles) or
// carried (carry_tile).  These are the tiled kernels' own functions in their
// order, so every result is bit-identical to the tiled path's; the two
// launches and the last-block hand-offs of every step disappear.
// Every CTA stores its tile partials (M, S, Q) into every CTA's shared memory
// (distributed shared memory) before the step's first cluster barrier; after
// it, every CTA combines the same partials with the same code, so each takes
// the same decisions in its own copy of the control block and finds its own
// tile's place in the cumulative weights, with no second barrier and no
// hand-off from one CTA to the others.  CTA 0 alone keeps the global copies
// (tile and group partials, control block) up to date.  The second barrier
// of the step orders the ancestors each CTA writes for the others' targets
// before the next step's gathers.
template <int KIND, int N, typename R>
__global__ void __launch_bounds__(TILE) k_filter_cluster(const FilterDev* __restrict__ fds,
                                                         const int* __restrict__ list, int cs_size) {
  __shared__ CombineScratch cs;
  __shared__ double ys[64];
  __shared__ Ctl sctl;          // this CTA's copy of the control block
  __shared__ TileTriples tri;   // the tile partials of the cluster's tiles
  __shared__ int s_lo, s_hi, nlong;
  __shared__ int s_nlast[WARPS];
  __shared__ double s_e0, s_scale_r, s_u;
  __shared__ int3 longr[TILE];
  const FilterDev& fd = fds[list[blockIdx.x / cs_size]];
  const int t = blockIdx.x % cs_size;
  const int tid = threadIdx.x;
  const int P = fd.P, T = fd.T, rs = fd.resampler;
  const bool mine = t < fd.ntiles;
  if (mine) init_tile<KIND, N, R>(fd, t);
  cluster_sync();
  if (tid == 0) {  // the initial control block, once from global memory
    const uint4* src = reinterpret_cast<const uint4*>(fd.ctl);
    uint4* dst = reinterpret_cast<uint4*>(&sctl);
    for (int k = 0; k < int(sizeof(Ctl) / sizeof(uint4)); ++k) dst[k] = ldcg(src + k);
  }
  __syncthreads();
  for (int i = 1; i <= T; ++i) {
    if (sctl.status != ST_OK || sctl.step != i) break;  // a degenerate step ended the run
    // the step's resampling uniform, drawn by the last thread while the others
    // gather and propagate (off the combine's serial path)
    if (tid == TILE - 1) s_u = resample_uniform(fd, i);
    if (mine) {
      const int j = t * TILE + tid;
      const int a_spec = (j < P && !fd.hist) ? fd.anc[j] : j;
      propagate_tile<KIND, N, R>(fd, t, i, sctl.anc_identity, sctl.lam_zero, sctl.cw, a_spec, ys,
                                 cs, &tri, cs_size);
    }
    cluster_sync();  // the tile partials of every CTA, in every CTA's shared memory
    const bool first = t == 0;
    constexpr bool OWN = OwnCombineMath<KIND, N>::value;
    if (combine_group<true, OWN>(fd, 0, cs, &tri, first))
      combine_filter<true, OWN>(fd, i, cs, &sctl, first, &s_u);
    __syncthreads();  // thread 0's decisions in sctl, the tiles' g and base in cs
    const bool go = sctl.status == ST_OK && sctl.rs_step == i && i < T && sctl.step == i + 1;
    if (tid == 0) nlong = 0;
    if (go && mine) {
      if (!sctl.rs_flag) {
        carry_tile(fd, t, i, sctl.M);
      } else {
        const int j = t * TILE + tid;
        const double ct = j < P ? fd.ctil[j] : 0.0;
        const double u = rs == RS_SYSTEMATIC ? sctl.u : 0.0;
        if (tid == 0 || tid == 32) {
          // this tile's place (what tile_base reads from the global partials):
          // base fma(G, base_t, 0), scale G g_t; the next tile's base, or S
          const double G = cs.G;
          const double base = tid == 0 ? fma(G, cs.tbase[t], 0.0)
                                       : (t + 1 < fd.ntiles ? fma(G, cs.tbase[t + 1], 0.0) : sctl.S);
          const int n0 = range_count(fd, rs, base, sctl.ratio, u, i);
          if (tid == 0) {
            s_e0 = base * sctl.ratio - u;
            s_scale_r = (G * cs.tg[t]) * sctl.ratio;
            s_lo = n0;
          } else {
            s_hi = n0;
          }
        }
        __syncthreads();
        resample_particles(fd, t, i, rs, s_lo, s_hi, s_e0, s_scale_r, ct, s_nlast, &nlong, longr);
      }
    }
    cluster_sync();  // the ancestors and carried weights of the next step
  }
}

// ---------------------------------------------------------------------------
// The batched form's persistent launch: one grid of resident CTAs works off a
// device queue of (filter, phase, tiles) items until every listed filter has
// run all its steps.
// ---------------------------------------------------------------------------
// A CTA takes the first slot of the highest-priority level that has one
// reserved, waits until it is filled, and processes
// the item with the tiled kernels' own functions, in their order: for a
// propagate item propagate_tile and, in the CTA that finishes the step's last
// tile (the tickets gp[g].ticket and gticket), the group and filter combines;
// for a resample item the per-tile resampling of k_resample (or the carry of
// the weights).  So every filter's results are bit-identical to the per-step
// launches'.  The CTA that finishes a phase pushes the filter's next one: its
// resample items after the combine, its propagate items of the next step after
// the last resampled tile (rticket).  A propagate item covers kt tiles, a
// resample item RS_CHUNK tiles (k_resample's chunk).  A filter of at most kt
// tiles is one item per phase, and the CTA that holds it goes on with the next
// phase itself, without the queue: its whole run stays on that CTA.
//
// Priority: the levels order items by their filter's remaining phases, the
// longest remaining runs first.  With one first-in-first-out queue every
// filter advanced one phase per pass through the whole queue, so the longest
// runs of a batch were the last to finish, alone on an idle GPU.
//
// No CTA waits while it holds work: a CTA waits only between items, for a
// slot it has taken (a race with another CTA can take a slot not yet
// reserved, which then waits for the level's next push), and every slot
// below a level's final total is filled by a CTA that is processing an item.
// So the run completes whatever the number of resident CTAs; a CTA ends when
// every level's items are taken.  Every wait is bounded (g_persist_wait_ns on
// the global timer); a wait that runs out sets err, and the other CTAs stop
// at their next wait.
//
// Memory ordering: a tile's writes are released by its ticket (the block's
// barrier, then a fence and the atomic) and a phase's by the push (the
// block's barrier, then st.release of each slot); the thread that takes a
// slot acquires it (ld.acquire) and the block's barrier passes that on to the
// other threads before they read anything the item depends on.
//
// Latency: a take reads every level's counters at once (relaxed loads, one
// round trip) and skips the levels this CTA has seen fully taken.  No slot
// is claimed ahead of the current item's end: a slot claimed early waits for
// the claiming CTA's item, which lengthened the longest runs' step chains
// more than the overlap saved.
// How long a wait may last (global-timer ns): 4 s unless a test shortens it.
__device__ unsigned long long g_persist_wait_ns = 4000000000ull;

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ int ld_relaxed_s32(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
// Record a failure of this run (err) and of the plan's runs so far (err_any).
__device__ __forceinline__ void persist_fail(PersistQueue* q, int code) {
  atomicExch(&q->err, code);
  atomicExch(&q->err_any, code);
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// The item in slot idx of level L once it is filled (acquired); 0 when the
// level gets no item idx (its total fell below idx) or the run has failed.
// The counters are read relaxed: only the slot itself synchronizes with the
// push that fills it.
__device__ unsigned long long persist_wait(PersistQueue* q, PersistLevel& L,
                                           const unsigned long long* slots,
                                           unsigned long long idx) {
  const unsigned long long t0 = global_ns();
  unsigned ns = 32;
  for (;;) {
    if (idx >= ld_relaxed_u64(&L.total)) return 0ull;
    const unsigned long long v = ld_acquire_u64(&slots[L.base + idx]);
    if (v != 0ull) return v;
    if (ld_relaxed_s32(&q->err) != 0) return 0ull;
    if (global_ns() - t0 > g_persist_wait_ns) {
      persist_fail(q, 1);
      return 0ull;
    }
    __nanosleep(ns);
    if (ns < 256) ns <<= 1;
  }
}

// Claim (thread 0) the first reserved slot of the highest-priority level that
// has one: its level, its index in *idx; -1 when no level has a reserved slot
// now, with *all_taken set when every level's items are taken.  The levels'
// counters are read together (relaxed loads, one round trip); `closed` keeps
// the levels this CTA found fully taken (head only grows and total only
// falls, so they stay so).
__device__ int persist_claim(PersistQueue* q, unsigned& closed, unsigned long long* idx,
                             bool* all_taken) {
  unsigned long long h[PERSIST_LEVELS], tot[PERSIST_LEVELS], tl[PERSIST_LEVELS];
#pragma unroll
  for (int l = 0; l < PERSIST_LEVELS; ++l) {
    h[l] = 0ull;
    tot[l] = 0ull;
    tl[l] = 0ull;
    if (!((closed >> l) & 1u)) {
      h[l] = ld_relaxed_u64(&q->lv[l].head);
      tot[l] = ld_relaxed_u64(&q->lv[l].total);
      tl[l] = ld_relaxed_u64(&q->lv[l].tail);
    }
  }
  *all_taken = true;
#pragma unroll
  for (int l = PERSIST_LEVELS - 1; l >= 0; --l) {
    if ((closed >> l) & 1u) continue;
    if (h[l] >= tot[l]) {
      closed |= 1u << l;
      continue;
    }
    *all_taken = false;
    if (h[l] < tl[l]) {
      *idx = atomicAdd(&q->lv[l].head, 1ull);
      return l;
    }
  }
  return -1;
}

// This CTA's next item (thread 0): claims and waits until one is filled; 0
// once every level's items are taken (the run is over) or the run has failed.
__device__ unsigned long long persist_take(PersistQueue* q, const unsigned long long* slots,
                                           unsigned& closed) {
  const unsigned long long t0 = global_ns();
  unsigned ns = 32;
  for (;;) {
    unsigned long long idx = 0;
    bool all_taken = false;
    const int l = persist_claim(q, closed, &idx, &all_taken);
    if (l >= 0) {
      const unsigned long long v = persist_wait(q, q->lv[l], slots, idx);
      if (v != 0ull) return v;
      if (ld_relaxed_s32(&q->err) != 0) return 0ull;
      continue;  // the level's total fell below the claimed slot: look again
    }
    if (all_taken || ld_relaxed_s32(&q->err) != 0) return 0ull;
    if (global_ns() - t0 > g_persist_wait_ns) {
      persist_fail(q, 1);
      return 0ull;
    }
    __nanosleep(ns);
    if (ns < 512) ns <<= 1;
  }
}

struct PersistShared {
  CombineScratch cs;
  double ys[64];
  unsigned long long item, next, base;
  int last, cont;
  RsChunk rc;  // resample items
};

// Fill n slots of level `level` with the items (k, phase, 0..n-1).  Every
// thread of the block calls it; the barrier orders the block's writes before
// the releases.
__device__ void persist_push(PersistQueue* q, unsigned long long* slots, int k, int phase, int n,
                             int level, PersistShared& sh) {
  PersistLevel& L = q->lv[level];
  __syncthreads();
  if (threadIdx.x == 0) sh.base = atomicAdd(&L.tail, static_cast<unsigned long long>(n));
  __syncthreads();
  const unsigned long long b = sh.base;
  if (b + static_cast<unsigned long long>(n) > L.cap) {
    // the plan's count rules this out; refuse rather than write past the level
    if (threadIdx.x == 0) persist_fail(q, 2);
    return;
  }
  for (int r = threadIdx.x; r < n; r += TILE)
    st_release_u64(&slots[L.base + b + r], persist_item(k, phase, r));
}

// Propagate item: tiles [qi kt, (qi + 1) kt) of filter k at its current step.
template <int KIND, int N, typename R>
__device__ void persist_propagate(const FilterDev& fd, int k, int qi, int kt, PersistQueue* q,
                                  unsigned long long* slots, PersistShared& sh) {
  const int tid = threadIdx.x;
  const int t0 = qi * kt, t1 = min(t0 + kt, fd.ntiles);
  // every thread reads the control block (L2) with its first tile's ancestor
  // row entry, so the two loads overlap
  const Ctl* ctl = fd.ctl;
  const int j0 = t0 * TILE + tid;
  int a_spec = (j0 < fd.P && !fd.hist) ? fd.anc[j0] : j0;
  const int i = ldcg(&ctl->step);
  const bool ok = ldcg(&ctl->status) == ST_OK;
  const int anc_identity = ldcg(&ctl->anc_identity);
  const int lam_zero = ldcg(&ctl->lam_zero);
  const double cw = ldcg(&ctl->cw);
  if (i > fd.T || !ok) {  // items are pushed only for running filters
    if (tid == 0) persist_fail(q, 3);
    return;
  }
  constexpr bool WARP = !(l96_kind(KIND) && N >= 16);
  constexpr bool OWN = OwnCombineMath<KIND, N>::value;
  bool finished = false;
  for (int t = t0; t < t1; ++t) {
    const int j = t * TILE + tid;
    if (t > t0) a_spec = (j < fd.P && !fd.hist) ? fd.anc[j] : j;
    propagate_tile<KIND, N, R>(fd, t, i, anc_identity, lam_zero, cw, a_spec, sh.ys, sh.cs);
    __syncthreads();  // the tile's states, prefixes and partials, before its ticket
    if (tid == 0) {
      __threadfence();
      const int g = t / GROUP;
      const int ntg = min(GROUP, fd.ntiles - g * GROUP);
      sh.last = atomicAdd(&fd.gp[g].ticket, 1u) == unsigned(ntg - 1);
    }
    __syncthreads();
    if (sh.last) {
      __threadfence();
      if (combine_group<WARP, OWN>(fd, t / GROUP, sh.cs)) {
        combine_filter<WARP, OWN>(fd, i, sh.cs);
        finished = true;
      }
    }
  }
  if (!finished) return;  // uniform over the block
  __syncthreads();        // thread 0's decisions in the control block
  const int nR = (fd.ntiles + RS_CHUNK - 1) / RS_CHUNK;
  if (tid == 0) {
    const Ctl* c = fd.ctl;  // written by this thread
    sh.cont = c->status == ST_OK && c->step == i + 1 && i < fd.T;
    // a filter that ends before its last step fills none of the slots of
    // its remaining phases: propagate at steps i+1..T, resample at i..T-1
    if (!sh.cont && i < fd.T && fd.ntiles > kt) {
      const long long nP = (fd.ntiles + kt - 1) / kt;
      for (int i2 = i + 1; i2 <= fd.T; ++i2)
        atomicAdd(&q->lv[persist_level(fd.T - i2 + 1, q->maxT)].total,
                  static_cast<unsigned long long>(-nP));
      for (int i2 = i; i2 < fd.T; ++i2)
        atomicAdd(&q->lv[persist_level(fd.T - i2, q->maxT)].total,
                  static_cast<unsigned long long>(-static_cast<long long>(nR)));
    }
  }
  __syncthreads();
  if (!sh.cont) return;
  if (fd.ntiles <= kt) {
    if (tid == 0) sh.next = persist_item(k, PHASE_RS, 0);
  } else {
    persist_push(q, slots, k, PHASE_RS, nR, persist_level(fd.T - i, q->maxT), sh);
  }
}

// Resample item: tiles [qi RS_CHUNK, (qi + 1) RS_CHUNK) of filter k after its
// current step, or all its tiles for a filter run whole on this CTA, in
// k_resample's chunks (resample_chunk: the same computation).
__device__ void persist_resample(const FilterDev* __restrict__ fds, int k, int qi, int kt,
                                 PersistQueue* q, unsigned long long* slots, PersistShared& sh) {
  const int tid = threadIdx.x;
  const FilterDev& fd = fds[k];
  const bool whole = fd.ntiles <= kt;
  const int t0 = whole ? 0 : qi * RS_CHUNK;
  const int t1 = whole ? fd.ntiles : min(t0 + RS_CHUNK, fd.ntiles);
  for (int c0 = t0; c0 < t1; c0 += RS_CHUNK)
    resample_chunk(fds, [&](int m) { return make_int2(k, c0 + m); }, min(RS_CHUNK, t1 - c0),
                   sh.rc);
  // resample_chunk ended with the block's barrier: the tiles' ancestors (or
  // carried weights) are written before the ticket
  if (tid == 0) {
    __threadfence();
    const unsigned n = unsigned(t1 - t0);
    sh.last = atomicAdd(&fd.ctl->rticket, n) == unsigned(fd.ntiles) - n;
  }
  __syncthreads();
  if (!sh.last) return;
  __threadfence();
  if (tid == 0) fd.ctl->rticket = 0u;  // for the next step (ordered by the push)
  if (whole) {
    if (tid == 0) sh.next = persist_item(k, PHASE_PROP, 0);
  } else {  // the next step's items: T - i propagate phases left
    persist_push(q, slots, k, PHASE_PROP, (fd.ntiles + kt - 1) / kt,
                 persist_level(fd.T - sh.rc.i[0], q->maxT), sh);
  }
}

// Blocks per SM the persistent kernel is compiled for: that of its largest
// class's propagate kernel (registers without spills); the sets with the FP32
// Lorenz '96 state are also compiled for four (64 registers, a few words
// spilled), which the launch takes when asked for four CTAs per SM.
template <int SET>
struct PersistOccupancy {
  static constexpr int value = (SET & PC_L8_64) ? 2 : (SET & PC_L8_32) ? 3 : 4;
};

template <int SET, int MINB>
__global__ void __launch_bounds__(TILE, MINB)
    k_persist(const FilterDev* __restrict__ fds, PersistQueue* q, unsigned long long* slots,
              int kt) {
  __shared__ PersistShared sh;
  const int tid = threadIdx.x;
  if (tid == 0) sh.next = 0ull;
  unsigned closed = 0u;  // thread 0: the levels found fully taken
  for (;;) {
    __syncthreads();  // the previous item's shared values are consumed
    if (tid == 0) {
      unsigned long long it = sh.next;
      sh.next = 0ull;
      if (it == 0ull) it = persist_take(q, slots, closed);  // acquires the slot
      sh.item = it;
    }
    __syncthreads();
    const unsigned long long it = sh.item;
    if (it == 0ull) return;
    const int k = int(it >> 32) - 1;
    const int phase = int((it >> 24) & 0xffu);
    const int qi = int(it & 0xffffffu);
    const FilterDev& fd = fds[k];
    if (phase == PHASE_RS) {
      persist_resample(fds, k, qi, kt, q, slots, sh);
      continue;
    }
    const bool dp = fd.prec == PREC_FP64;
    if constexpr ((SET & PC_WK64) != 0) {
      if (fd.kind == KIND_WK && dp) {
        persist_propagate<KIND_WK, 1, double>(fd, k, qi, kt, q, slots, sh);
        continue;
      }
    }
    if constexpr ((SET & PC_WK32) != 0) {
      if (fd.kind == KIND_WK && !dp) {
        persist_propagate<KIND_WK, 1, float>(fd, k, qi, kt, q, slots, sh);
        continue;
      }
    }
    if constexpr ((SET & PC_L8_64) != 0) {
      if (fd.kind == KIND_L96 && fd.N == 8 && dp) {
        persist_propagate<KIND_L96, 8, double>(fd, k, qi, kt, q, slots, sh);
        continue;
      }
    }
    if constexpr ((SET & PC_L8_32) != 0) {
      if (fd.kind == KIND_L96 && fd.N == 8 && !dp) {
        persist_propagate<KIND_L96, 8, float>(fd, k, qi, kt, q, slots, sh);
        continue;
      }
    }
    if (tid == 0) persist_fail(q, 3);  // a class outside the set: never queued by a plan
    return;
  }
}

// ---------------------------------------------------------------------------
// Multinomial resampling: the spacings of the sorted uniforms
// ---------------------------------------------------------------------------
// After the propagate launch of step i (rs_step = i), for every filter that
// resamples with the multinomial scheme: unit exponentials e_l = -log v_l
// (v_l in (0, 1] from Philox block (l, i, RESAMPLE, 2)), l = 0..P; their
// in-tile inclusive sums go to mn_t, the tile totals to mn_part.
__device__ __forceinline__ bool mn_active(const FilterDev& fd, int* step) {
  const Ctl* c = fd.ctl;
  const int i0 = ldcg(&c->rs_step);
  *step = i0;
  return fd.resampler == RS_MULTINOMIAL && ldcg(&c->status) == ST_OK && i0 >= 1 && i0 < fd.T &&
         ldcg(&c->step) == i0 + 1 && ldcg(&c->rs_flag) != 0;
}

// Spacing l: -log v in FP64 (own log), v in (0, 1] the 53-bit uniform of
// words 1:0 of block (l, i, RESAMPLE, 2).
__device__ __forceinline__ double mn_spacing(const FilterDev& fd, int l, int i) {
  const uint4 w = rng_block(fd.seed, uint32_t(l), uint32_t(i), PURPOSE_RESAMPLE, 2u);
  return -log_pos(u53_open_closed(w.x, w.y));
}

__global__ void __launch_bounds__(TILE) k_mn_tiles(const FilterDev* __restrict__ fds,
                                                   const int2* __restrict__ tmap) {
  __shared__ BlockScratch b;
  __shared__ int s_go, s_i;
  const int2 ft = tmap[blockIdx.x];
  const FilterDev& fd = fds[ft.x];
  if (fd.resampler != RS_MULTINOMIAL) return;
  if (threadIdx.x == 0) s_go = mn_active(fd, &s_i);
  __syncthreads();
  if (!s_go) return;
  const int l = ft.y * TILE + threadIdx.x;
  const double e = l < fd.P ? mn_spacing(fd, l, s_i) : 0.0;
  double tot;
  const double incl = block_scan(e, b, &tot);
  if (l < fd.P) fd.mn_t[l] = incl;
  if (threadIdx.x == 0) fd.mn_part[ft.y] = tot;
}

// One block per filter: exclusive scan of the tile totals in place, then
// mn_part[ntiles] = P / (all P + 1 spacings).
__global__ void __launch_bounds__(TILE) k_mn_total(const FilterDev* __restrict__ fds, int nf) {
  __shared__ BlockScratch b;
  __shared__ int s_go, s_i;
  const FilterDev& fd = fds[blockIdx.x];
  if (fd.resampler != RS_MULTINOMIAL || fd.ctl == nullptr) return;
  if (threadIdx.x == 0) s_go = mn_active(fd, &s_i);
  __syncthreads();
  if (!s_go) return;
  const int nt = fd.ntiles;
  const int chunk = (nt + TILE - 1) / TILE;
  const int lo = min(nt, int(threadIdx.x) * chunk), hi = min(nt, lo + chunk);
  double s = 0.0;
  for (int q = lo; q < hi; ++q) s += fd.mn_part[q];
  double tot;
  const double incl = block_scan(s, b, &tot);
  double run = incl - s;
  for (int q = lo; q < hi; ++q) {
    const double v = fd.mn_part[q];
    fd.mn_part[q] = run;
    run += v;
  }
  if (threadIdx.x == 0) fd.mn_part[nt] = double(fd.P) / (tot + mn_spacing(fd, fd.P, s_i));
}

// Scaled targets in place: mn_t[l] = (tile offset + in-tile sum) P / total.
__global__ void __launch_bounds__(TILE) k_mn_targets(const FilterDev* __restrict__ fds,
                                                     const int2* __restrict__ tmap) {
  __shared__ int s_go, s_i;
  const int2 ft = tmap[blockIdx.x];
  const FilterDev& fd = fds[ft.x];
  if (fd.resampler != RS_MULTINOMIAL) return;
  if (threadIdx.x == 0) s_go = mn_active(fd, &s_i);
  __syncthreads();
  if (!s_go) return;
  const int l = ft.y * TILE + threadIdx.x;
  if (l < fd.P)
    fd.mn_t[l] = (ldcg(&fd.mn_part[ft.y]) + fd.mn_t[l]) * ldcg(&fd.mn_part[fd.ntiles]);
}

// ---------------------------------------------------------------------------
// Single state path (end of Algorithm 2)
// ---------------------------------------------------------------------------
// Draw one particle from the final weights of filter 0: the first k whose
// scaled cumulative weight C_k (P / S) exceeds v P, with v the uniform of the
// path purpose at step T + 1.  Each tile evaluates C_k (P / S) as the
// resampling kernel does (with u = 0) and offers its first qualifying
// particle to an atomic minimum in *pick (set to a large value beforehand).
__global__ void __launch_bounds__(TILE) k_path_pick(const FilterDev* __restrict__ fds,
                                                    int32_t* __restrict__ pick) {
  const FilterDev& fd = fds[0];
  const int t = blockIdx.x;
  const int tid = threadIdx.x;
  const int P = fd.P;
  const int j0 = t * TILE;
  const int g = t / GROUP;
  const double ct = j0 + tid < P ? fd.ctil[j0 + tid] : 0.0;
  const double gG = fd.gp[g].G, gB = fd.gp[g].B, tbase = fd.tp[t].base, tg = fd.tp[t].g;
  __shared__ int s_ok, s_first;
  __shared__ double s_ratio, s_tau;
  if (tid == 0) {
    const Ctl* c = fd.ctl;
    s_ok = ldcg(&c->status) == ST_OK && ldcg(&c->step) == fd.T + 1;
    s_ratio = double(P) / ldcg(&c->S);
    const uint4 w = rng_block(fd.seed, 0u, uint32_t(fd.T + 1), PURPOSE_PATH, 0u);
    s_tau = u53_closed_open(w.x, w.y) * double(P);
    s_first = TILE;
  }
  __syncthreads();
  if (!s_ok) return;
  const double ratio = s_ratio;
  const double e0 = fma(gG, tbase, gB) * ratio;
  const double scale_r = (gG * tg) * ratio;
  if (j0 + tid < P && fma(scale_r, ct, e0) > s_tau) atomicMin(&s_first, tid);
  __syncthreads();
  if (tid == 0 && s_first < TILE) atomicMin(pick, j0 + s_first);
}

// Follow the ancestor history of filter 0 back from the picked particle:
// b_T = pick (clamped to P - 1 when no cumulative weight exceeded the target),
// b_{i-1} = a(t_i)[b_i].  One thread; idx[T] holds the pick on entry.  A
// degenerate filter gives idx = -1 everywhere.
__global__ void k_path_trace(const FilterDev* __restrict__ fds, int32_t* __restrict__ idx) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  const FilterDev& fd = fds[0];
  const int P = fd.P, T = fd.T;
  if (ldcg(&fd.ctl->status) != ST_OK || !fd.hist) {
    for (int i = 0; i <= T; ++i) idx[i] = -1;
    return;
  }
  int b = min(idx[T], P - 1);
  idx[T] = b;
  for (int i = T; i >= 1; --i) {
    b = (b >= 0 && b < P) ? fd.anc[int64_t(i - 1) * P + b] : -1;
    idx[i - 1] = b;
  }
}

// path[i][n] = x(t_i)[n][idx[i]] in FP64 (N threads); NaN when idx[i] is not a particle.
__global__ void k_path_copy(const void* __restrict__ x, int prec, int N, int P,
                            const int32_t* __restrict__ idx, int i, double* __restrict__ path) {
  const int n = threadIdx.x;
  if (n >= N) return;
  const int b = idx[i];
  double v = NAN;
  if (b >= 0 && b < P) {
    const int64_t at = int64_t(n) * P + b;
    v = prec == PREC_MIXED ? double(static_cast<const float*>(x)[at])
                         : static_cast<const double*>(x)[at];
  }
  path[int64_t(i) * N + n] = v;
}

// The normals of the FP64 windkessel transition of filter fds[k] for steps
// first..last, drawn ahead into its table: znoise[(i - 1) s + mm][j] is normal
// number mm of stream (j, i, PROP), from the same Philox block and Box-Muller
// pair as the propagate kernel would draw.  One thread per particle and pair
// of substeps, over the whole GPU: a small filter's propagation then reads
// its normals instead of spending B300's FP64 unit (1/64 of the FP32 rate)
// on them in the few SMs its tiles occupy.  The key is read from the device
// descriptor, so samplers that rewrite it on the device get their own draws.
__global__ void k_noise_wk64(const FilterDev* __restrict__ fds, int k, int first, int last) {
  const FilterDev& fd = fds[k];
  const int P = fd.P, s = fd.s, hb = (s + 1) / 2;
  const uint64_t seed = fd.seed;
  double* zt = const_cast<double*>(fd.znoise);
  const int64_t n = int64_t(last - first + 1) * hb * P;
  for (int64_t q = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; q < n;
       q += int64_t(gridDim.x) * blockDim.x) {
    const int j = int(q % P);
    const int64_t r = q / P;
    const int b = int(r % hb);
    const int i = first + int(r / hb);
    double z0, z1;
    normal_pair64(rng_block(seed, uint32_t(j), uint32_t(i), PURPOSE_PROP, uint32_t(b)), &z0, &z1);
    double* zr = zt + (int64_t(i - 1) * s + 2 * b) * P + j;
    zr[0] = z0;
    if (2 * b + 1 < s) zr[P] = z1;
  }
}

// Windkessel input table F(k dt), k < n: half sine of the given peak and period.
__global__ void k_flow(double* __restrict__ flow, int64_t n, double peak, double period,
                       double dt) {
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const double t = double(k) * dt;
  const double ph = t / period;
  const double fr = ph - floor(ph);
  double v = 0.0;
  if (fr < 0.5) {
    double sn, cs;
    sincos_2pi(fr, &sn, &cs);
    v = peak * sn;
  }
  flow[k] = v;
}

// Filter fds[0] about to propagate to t_step from a state loaded from outside
// (a diagnostic for teacher-forced checks): the control block as after a
// resampling (carried log-weights zero, no likelihood accumulated yet),
// ancestors from the array or the identity, group tickets cleared.
__global__ void k_debug_ctl(const FilterDev* __restrict__ fds, int step, int anc_identity) {
  const FilterDev& fd = fds[0];
  if (threadIdx.x == 0) {
    Ctl* c = fd.ctl;
    const double r = wk_kind(fd.kind) ? fd.theta[4] : fd.theta[2];
    c->step = step;
    c->rs_step = step - 1;
    c->rs_flag = 0;
    c->anc_identity = anc_identity;
    c->lam_zero = 1;
    c->status = ST_OK;
    c->gticket = 0u;
    c->rticket = 0u;
    c->ll = 0.0;
    c->logP = log(double(fd.P));
    c->L = c->logP;
    c->c_obs = -0.5 * double(fd.Ny) * log(2.0 * 3.141592653589793 * r);
    c->cw = -0.5 / r;
    c->M = 0.0;
    c->S = 0.0;
    c->u = 0.0;
    c->ratio = 0.0;
    if (l96_kind(fd.kind)) l96_constants32(fd, c->lf);
  }
  for (int g = threadIdx.x; g < fd.ngroups; g += blockDim.x) fd.gp[g].ticket = 0u;
  for (int t = threadIdx.x; t < fd.ntiles; t += blockDim.x) fd.tp[t].ticket = 0u;
}

// The ancestors the next propagation of filter fds[0] takes (diagnostic): the
// array the resample kernel wrote, or the identity after a step that carried
// its weights; nothing once the filter has finished or degenerated.
__global__ void k_next_ancestors(const FilterDev* __restrict__ fds, int32_t* __restrict__ out) {
  const FilterDev& fd = fds[0];
  const Ctl* c = fd.ctl;
  if (ldcg(&c->status) != ST_OK || ldcg(&c->step) > fd.T) return;
  const int identity = ldcg(&c->anc_identity);
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < fd.P) out[j] = identity ? j : fd.anc[j];
}

// Copy (loglik, status, next step) of nf filters into out[3k .. 3k+2];
// descriptors without a control block (empty server slots) give NaNs.
__global__ void k_results(const FilterDev* __restrict__ fds, int nf, double* __restrict__ out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nf) return;
  const Ctl* c = fds[k].ctl;
  if (c == nullptr) {
    out[3 * k] = out[3 * k + 1] = out[3 * k + 2] = NAN;
    return;
  }
  out[3 * k] = ldcg(&c->ll);
  out[3 * k + 1] = double(ldcg(&c->status));
  out[3 * k + 2] = double(ldcg(&c->step));
}

// ---------------------------------------------------------------------------
// Host-side dispatch
// ---------------------------------------------------------------------------
#define PF_L96_SIZES(X) X(4) X(8) X(12) X(16) X(20) X(24) X(32) X(40)

bool supported(int kind, int N, int prec) {
  if (prec != PREC_FP64 && prec != PREC_MIXED) return false;
  if (wk_kind(kind)) return N == 1;
  if (!l96_kind(kind)) return false;
#define PF_CASE(n) if (N == n) return true;
  PF_L96_SIZES(PF_CASE)
#undef PF_CASE
  return false;
}

enum { LAUNCH_INIT = 0, LAUNCH_PROPAGATE = 1, LAUNCH_CTA = 2 };

// Launch with programmatic stream serialization (see wait_prior_grid): the
// launch of a step kernel overlaps the drain of the one before it.
template <typename... Params, typename... Args>
static cudaError_t launch_chained(void (*kernel)(Params...), unsigned grid, cudaStream_t st,
                                  Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(TILE);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

template <int KIND, int N, typename R>
static cudaError_t launch_pair(int what, const FilterDev* fds, const int2* tmap, int nblocks,
                               cudaStream_t st) {
  if (nblocks <= 0) return cudaSuccess;
  if (what == LAUNCH_INIT) {
    k_init<KIND, N, R><<<nblocks, TILE, 0, st>>>(fds, tmap);
  } else if (what == LAUNCH_PROPAGATE) {
    const cudaError_t e =
        launch_chained(k_propagate<KIND, N, R>, unsigned(nblocks), st, fds, tmap);
    if (e != cudaSuccess) return e;
  } else {
    // nblocks = filters x cluster size, what - LAUNCH_CTA = the cluster size
    const int cs_size = what - LAUNCH_CTA;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(unsigned(nblocks));
    cfg.blockDim = dim3(TILE);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = unsigned(cs_size);
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const cudaError_t e = cudaLaunchKernelEx(&cfg, k_filter_cluster<KIND, N, R>, fds,
                                             reinterpret_cast<const int*>(tmap), cs_size);
    if (e != cudaSuccess) return e;
  }
  return cudaGetLastError();
}

static cudaError_t dispatch(int init, int kind, int N, int prec, const FilterDev* fds,
                            const int2* tmap, int nblocks, cudaStream_t st) {
  const bool dp = prec == PREC_FP64;
  if (kind == KIND_WK) {
    return dp ? launch_pair<KIND_WK, 1, double>(init, fds, tmap, nblocks, st)
              : launch_pair<KIND_WK, 1, float>(init, fds, tmap, nblocks, st);
  }
  if (kind == KIND_WKX) {
    return dp ? launch_pair<KIND_WKX, 1, double>(init, fds, tmap, nblocks, st)
              : launch_pair<KIND_WKX, 1, float>(init, fds, tmap, nblocks, st);
  }
  if (kind == KIND_L96) {
#define PF_CASE(n)                                                                       \
  if (N == n)                                                                            \
    return dp ? launch_pair<KIND_L96, n, double>(init, fds, tmap, nblocks, st)           \
              : launch_pair<KIND_L96, n, float>(init, fds, tmap, nblocks, st);
    PF_L96_SIZES(PF_CASE)
#undef PF_CASE
  }
  if (kind == KIND_L96W) {
#define PF_CASE(n)                                                                       \
  if (N == n)                                                                            \
    return dp ? launch_pair<KIND_L96W, n, double>(init, fds, tmap, nblocks, st)          \
              : launch_pair<KIND_L96W, n, float>(init, fds, tmap, nblocks, st);
    PF_L96_SIZES(PF_CASE)
#undef PF_CASE
  }
  return cudaErrorInvalidValue;
}

// The checked build's counters, then zeroed.
cudaError_t read_checks(unsigned long long* out) {
  cudaError_t e = cudaMemcpyFromSymbol(out, g_checks, sizeof(g_checks));
  if (e != cudaSuccess) return e;
  const unsigned long long zero[CHK_KINDS] = {};
  return cudaMemcpyToSymbol(g_checks, zero, sizeof(zero));
}

// The weight exponential on n given arguments (diagnostic entry point).
__global__ void k_weight_exp(const double* __restrict__ d, double* __restrict__ w, int64_t n) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n;
       i += int64_t(gridDim.x) * blockDim.x)
    w[i] = exp_weight(d[i]);
}

// The weight-sum logarithm on n given arguments (diagnostic entry point).
__global__ void k_log_sum(const double* __restrict__ s, double* __restrict__ y, int64_t n) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n;
       i += int64_t(gridDim.x) * blockDim.x)
    y[i] = log_sum(s[i]);
}

cudaError_t launch_log_sum(const double* s, double* y, int64_t n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int64_t nb = (n + TILE - 1) / TILE;
  k_log_sum<<<unsigned(nb < 4096 ? nb : 4096), TILE, 0, st>>>(s, y, n);
  return cudaGetLastError();
}

// The propagate kernels' in-tile prefix of given weights (tile_epilogue's
// weight_fixed / block_scan_fixed / fixed_double), one block per tile of
// TILE weights (past n: 0): prefix[j] for every j < n, total[t] per tile.
__global__ void __launch_bounds__(TILE) k_tile_prefix(const double* __restrict__ w,
                                                      double* __restrict__ prefix,
                                                      double* __restrict__ total, int64_t n) {
  __shared__ BlockScratch b;
  const int64_t j = int64_t(blockIdx.x) * TILE + threadIdx.x;
  const double v = j < n ? w[j] : 0.0;
  unsigned long long tot;
  const double c = fixed_double(block_scan_fixed(weight_fixed(v), b, &tot));
  if (j < n) prefix[j] = c;
  if (threadIdx.x == 0) total[blockIdx.x] = fixed_double(tot);
}

cudaError_t launch_tile_prefix(const double* w, double* prefix, double* total, int64_t n,
                               cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int64_t nb = (n + TILE - 1) / TILE;
  k_tile_prefix<<<unsigned(nb), TILE, 0, st>>>(w, prefix, total, n);
  return cudaGetLastError();
}

cudaError_t launch_weight_exp(const double* d, double* w, int64_t n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int64_t nb = (n + TILE - 1) / TILE;
  k_weight_exp<<<unsigned(nb < 4096 ? nb : 4096), TILE, 0, st>>>(d, w, n);
  return cudaGetLastError();
}

// The current device's SM count, queried once per process (a function-local
// static: its initialisation is thread-safe, so host threads launching at
// the same time see one value).
static int device_sms() {
  static const int sms = [] {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    return cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && n > 0
               ? n
               : 148;
  }();
  return sms;
}

// Blocks per tile of the sub-tile propagate launch for FP64 tiles of a plan
// of `ntiles` tiles in all: 4 or 2 when the state is FP64 and that many
// blocks per tile still fit the GPU's resident blocks at once, else 1
// (k_propagate).
template <int KIND, int N, typename R>
static int sub_for(int ntiles) {
  if constexpr (sizeof(R) != 8) {
    return 1;
  } else {
    const long long slots =
        static_cast<long long>(device_sms()) * PropagateOccupancy<KIND, N, R>::value;
    if (4ll * ntiles <= slots) return 4;
    if (2ll * ntiles <= slots) return 2;
    return 1;
  }
}

template <int KIND, int N, typename R>
static cudaError_t launch_sub(int sub, const FilterDev* fds, const int2* tmap, int ntiles,
                              cudaStream_t st) {
  if (ntiles <= 0) return cudaSuccess;
  cudaError_t e = cudaSuccess;
  if (sub == 4)
    e = launch_chained(k_propagate_sub<KIND, N, R, 4>, unsigned(4 * ntiles), st, fds, tmap);
  else if (sub == 2)
    e = launch_chained(k_propagate_sub<KIND, N, R, 2>, unsigned(2 * ntiles), st, fds, tmap);
  else
    e = launch_chained(k_propagate<KIND, N, R>, unsigned(ntiles), st, fds, tmap);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

// The classes with a sub-tile propagate kernel: FP64 Lorenz '96 (both forms)
// up to N = 12, whose RK4 substeps and normals make a tile's FP64 work long.
// The FP64 windkessel's step is too light: split, its tiles only lengthened
// each step's chain of dependent phases.
#define PF_SUB_CLASSES(X)                                                          \
  X(KIND_L96, 4) X(KIND_L96, 8) X(KIND_L96, 12) X(KIND_L96W, 4) X(KIND_L96W, 8)   \
  X(KIND_L96W, 12)

int propagate_sub(int kind, int N, int prec, int ntiles) {
  if (prec != PREC_FP64) return 1;
#define PF_CASE(k, n) \
  if (kind == k && N == n) return sub_for<k, n, double>(ntiles);
  PF_SUB_CLASSES(PF_CASE)
#undef PF_CASE
  return 1;
}

cudaError_t launch_propagate_sub(int kind, int N, int prec, int sub, const FilterDev* fds,
                                 const int2* tmap, int ntiles, cudaStream_t st) {
  if (sub <= 1 || prec != PREC_FP64) return launch_propagate(kind, N, prec, fds, tmap, ntiles, st);
#define PF_CASE(k, n) \
  if (kind == k && N == n) return launch_sub<k, n, double>(sub, fds, tmap, ntiles, st);
  PF_SUB_CLASSES(PF_CASE)
#undef PF_CASE
  return cudaErrorInvalidValue;
}

cudaError_t launch_init(int kind, int N, int prec, const FilterDev* fds, const int2* tmap,
                        int nblocks, cudaStream_t st) {
  return dispatch(LAUNCH_INIT, kind, N, prec, fds, tmap, nblocks, st);
}

cudaError_t launch_propagate(int kind, int N, int prec, const FilterDev* fds, const int2* tmap,
                             int nblocks, cudaStream_t st) {
  return dispatch(LAUNCH_PROPAGATE, kind, N, prec, fds, tmap, nblocks, st);
}

cudaError_t launch_filter_cluster(int kind, int N, int prec, const FilterDev* fds,
                                  const int* list, int nfilters, int cluster_size,
                                  cudaStream_t st) {
  if (cluster_size < 1 || cluster_size > MAX_CLUSTER_TILES) return cudaErrorInvalidValue;
  return dispatch(LAUNCH_CTA + cluster_size, kind, N, prec, fds,
                  reinterpret_cast<const int2*>(list), nfilters * cluster_size, st);
}

cudaError_t launch_resample(const FilterDev* fds, const int2* tmap, int nblocks,
                            cudaStream_t st, int blocks_per_sm) {
  if (nblocks <= 0) return cudaSuccess;
  const int sms = device_sms();
  const int bps = std::min(std::max(blocks_per_sm, 1), RESAMPLE_BLOCKS_PER_SM);
  const int grid = std::min(nblocks, sms * bps);
  const cudaError_t e = launch_chained(k_resample, unsigned(grid), st, fds, tmap, nblocks);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

cudaError_t set_persist_wait_limit(unsigned long long ns) {
  return cudaMemcpyToSymbol(g_persist_wait_ns, &ns, sizeof(ns));
}

int persist_class_bit(int kind, int N, int prec) {
  if (kind == KIND_WK && N == 1) return prec == PREC_FP64 ? PC_WK64 : PC_WK32;
  if (kind == KIND_L96 && N == 8) return prec == PREC_FP64 ? PC_L8_64 : PC_L8_32;
  return 0;
}

// The class sets the persistent kernel is compiled for: each model class
// alone, and the windkessel with Lorenz '96 N = 8 in one precision.
#define PF_PERSIST_SETS(X)                                                       \
  X(PC_WK64) X(PC_WK32) X(PC_L8_64) X(PC_L8_32) X(PC_WK64 | PC_L8_64) X(PC_WK32 | PC_L8_32)

bool persist_set_supported(int set) {
#define PF_CASE(m) if (set == (m)) return true;
  PF_PERSIST_SETS(PF_CASE)
#undef PF_CASE
  return false;
}

template <int SET, int MINB>
static cudaError_t launch_persist_occ(const FilterDev* fds, PersistQueue* q,
                                      unsigned long long* slots, int kt, int blocks_per_sm,
                                      cudaStream_t st) {
  const int sms = device_sms();
  static const int occ = [] {  // resident CTAs per SM, once per instantiation (thread-safe)
    int o = 0;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_persist<SET, MINB>, TILE, 0) ==
                       cudaSuccess && o >= 1
               ? o
               : 1;
  }();
  const int bps = std::min(std::max(blocks_per_sm, 1), occ);
  k_persist<SET, MINB><<<sms * bps, TILE, 0, st>>>(fds, q, slots, kt);
  return cudaGetLastError();
}

template <int SET>
static cudaError_t launch_persist_set(const FilterDev* fds, PersistQueue* q,
                                      unsigned long long* slots, int kt, int blocks_per_sm,
                                      cudaStream_t st) {
  constexpr int occ = PersistOccupancy<SET>::value;
  if constexpr (occ == 3) {
    if (blocks_per_sm >= 4)
      return launch_persist_occ<SET, 4>(fds, q, slots, kt, blocks_per_sm, st);
  }
  return launch_persist_occ<SET, occ>(fds, q, slots, kt, blocks_per_sm, st);
}

cudaError_t launch_persist(int set, const FilterDev* fds, PersistQueue* q,
                           unsigned long long* slots, int kt, int blocks_per_sm,
                           cudaStream_t st) {
  if (kt < 1 || kt > MAX_CLUSTER_TILES || (kt & (kt - 1)) != 0) return cudaErrorInvalidValue;
#define PF_CASE(m) \
  if (set == (m)) return launch_persist_set<(m)>(fds, q, slots, kt, blocks_per_sm, st);
  PF_PERSIST_SETS(PF_CASE)
#undef PF_CASE
  return cudaErrorInvalidValue;
}

cudaError_t launch_flow(double* flow, int64_t n, double peak, double period, double dt,
                        cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int bs = 256;
  k_flow<<<int((n + bs - 1) / bs), bs, 0, st>>>(flow, n, peak, period, dt);
  return cudaGetLastError();
}

cudaError_t launch_results(const FilterDev* fds, int nf, double* out, cudaStream_t st) {
  if (nf <= 0) return cudaSuccess;
  k_results<<<(nf + 127) / 128, 128, 0, st>>>(fds, nf, out);
  return cudaGetLastError();
}

cudaError_t launch_mn_scan(const FilterDev* fds, const int2* tmap, int ntiles, int nf,
                           cudaStream_t st) {
  if (ntiles <= 0) return cudaSuccess;
  k_mn_tiles<<<ntiles, TILE, 0, st>>>(fds, tmap);
  k_mn_total<<<nf, TILE, 0, st>>>(fds, nf);
  k_mn_targets<<<ntiles, TILE, 0, st>>>(fds, tmap);
  return cudaGetLastError();
}

cudaError_t launch_noise(const FilterDev* fds, int k, int first, int last, int P, int s,
                         cudaStream_t st) {
  if (last < first) return cudaSuccess;
  const int sms = device_sms();
  const int64_t n = int64_t(last - first + 1) * ((s + 1) / 2) * P;
  const int64_t nb = (n + 255) / 256;
  k_noise_wk64<<<unsigned(std::min<int64_t>(nb, int64_t(sms) * 8)), 256, 0, st>>>(fds, k, first,
                                                                                  last);
  return cudaGetLastError();
}

cudaError_t launch_debug_ctl(const FilterDev* fds, int step, int anc_identity, cudaStream_t st) {
  k_debug_ctl<<<1, TILE, 0, st>>>(fds, step, anc_identity);
  return cudaGetLastError();
}

cudaError_t launch_next_ancestors(const FilterDev* fds, int ntiles, int32_t* out,
                                  cudaStream_t st) {
  if (ntiles <= 0) return cudaSuccess;
  k_next_ancestors<<<ntiles, TILE, 0, st>>>(fds, out);
  return cudaGetLastError();
}

cudaError_t launch_path_pick(const FilterDev* fds, int ntiles, int32_t* pick, cudaStream_t st) {
  k_path_pick<<<ntiles, TILE, 0, st>>>(fds, pick);
  return cudaGetLastError();
}

cudaError_t launch_path_trace(const FilterDev* fds, int32_t* idx, cudaStream_t st) {
  k_path_trace<<<1, 32, 0, st>>>(fds, idx);
  return cudaGetLastError();
}

cudaError_t launch_path_copy(const void* x, int prec, int N, int P, const int32_t* idx, int i,
                             double* path, cudaStream_t st) {
  k_path_copy<<<1, 64, 0, st>>>(x, prec, N, P, idx, i, path);
  return cudaGetLastError();
}

}  // namespace pfb
