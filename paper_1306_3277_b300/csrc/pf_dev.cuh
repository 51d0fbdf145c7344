// pf_dev.cuh -- device-side building blocks of the B300 bootstrap particle
// filter (arXiv 1306.3277, Algorithm 2): descriptors, Philox4x32-10,
// project-written log / sincos(2 pi u) for Box-Muller and exp for the exact
// windkessel, and the canonical block reductions and scans that fix the
// summation order of every run.
//
// The whole library is compiled with -fmad=false: a fused multiply-add
// happens only where the code calls fma()/fmaf(); every other operation is
// rounded on its own, so results are reproducible bit for bit.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace pfb {

constexpr int TILE = 256;        // particles per tile == threads per block
constexpr int GROUP = 256;       // tiles per group (two-level combine)
constexpr int WARPS = TILE / 32;
constexpr int64_t MAX_P = int64_t(1) << 24;  // GROUP * GROUP * TILE
constexpr int MAX_CLUSTER_TILES = 8;          // the portable thread-block cluster size
constexpr int RS_CHUNK = 4;   // tiles a resample block (or persistent resample item) takes at once

// Checked builds (-DPF_CHECKED=1, libpf_b300_checked.so) count violations of
// the path's invariants on the device instead of assuming them: an ancestor
// outside [0, P) (then replaced by the particle's own index, so every access
// stays in bounds), a non-finite propagated state, a decreasing in-tile
// cumulative weight, an offspring range that ends before it starts or leaves
// [0, P].  Nothing traps; pf_debug_check_counts reads the counts.
#ifndef PF_CHECKED
#define PF_CHECKED 0
#endif
enum { CHK_ANCESTOR = 0, CHK_STATE = 1, CHK_PREFIX = 2, CHK_RANGE = 3, CHK_KINDS = 4 };

enum { KIND_WK = 0, KIND_L96 = 1, KIND_WKX = 2, KIND_L96W = 3 };
__host__ __device__ constexpr bool wk_kind(int k) { return k == KIND_WK || k == KIND_WKX; }
__host__ __device__ constexpr bool l96_kind(int k) { return k == KIND_L96 || k == KIND_L96W; }
enum { PREC_FP64 = 0, PREC_MIXED = 1 };
enum { MODE_ALWAYS = 0, MODE_ADAPTIVE = 1, MODE_NEVER = 2 };
enum { RS_SYSTEMATIC = 0, RS_STRATIFIED = 1, RS_MULTINOMIAL = 2 };
enum { PURPOSE_INIT = 1, PURPOSE_PROP = 2, PURPOSE_RESAMPLE = 3, PURPOSE_PATH = 4 };
enum { ST_OK = 0, ST_DEGENERATE = 4 };

// Per tile of TILE particles: written by the propagate kernel (M, S, Q) and
// by the group combine (g, base).
struct alignas(16) TilePart {
  double M;     // max log-weight in the tile
  double S;     // sum exp(ell - M) over the tile (inclusive-scan total)
  double Q;     // sum exp(2 (ell - M)) (adaptive resampling only)
  double g;     // exp(M - M_group)
  double base;  // exclusive prefix of the scaled tile sums inside the group
  unsigned ticket;  // sub-tile propagate launch: parts of the tile finished this step
  unsigned pad;
};

struct alignas(16) GroupPart {
  double M, S, Q;   // group max, scaled sum, scaled square sum
  double G;         // exp(M_group - M_filter)
  double B;         // exclusive prefix of the scaled group sums
  unsigned ticket;  // tiles of this group finished in the current step
  unsigned pad0;
  double pad1, pad2;
};

// Per-filter control block, written by the last block of each propagate
// kernel and read by the next launches.
struct alignas(16) Ctl {
  int32_t step;          // next observation to propagate to (1..T; T+1 = done)
  int32_t rs_step;       // step whose resampling the resample kernel performs
  int32_t rs_flag;       // 1: resample at rs_step, 0: carry the weights
  int32_t anc_identity;  // propagate kernel: identity ancestors
  int32_t lam_zero;      // propagate kernel: carried log-weights are all zero
  int32_t status;        // ST_OK / ST_DEGENERATE
  uint32_t gticket;      // groups finished in the current step
  uint32_t rticket;      // persistent launch: tiles resampled in the current step
  double ll;             // log-likelihood accumulated so far
  double L;              // log sum_j exp(lam_j) of the carried log-weights
  double M, S;           // max and scaled sum of the current step
  double u;              // resampling uniform of the current step
  double ratio;          // P / S (systematic targets compared in the scaled form)
  double c_obs;          // -Ny/2 log(2 pi r)
  double logP;           // log P
  double cw;             // -0.5 / r: scale of the residual sum of squares
  float lf[6];           // FP32 Lorenz '96: F, dt, dt/2, dt/3, dt/6, sqrt(q) of the run
  float lpad[2];
};

// Descriptor of one filter (device copy read by every kernel).
struct alignas(16) FilterDev {
  int32_t kind, N, s, stride, prec, Ny;
  int32_t P, T, ntiles, ngroups, hist, mode;
  int32_t resampler;  // RS_*
  int32_t obs_every;  // >= 1: step i is observed iff i % obs_every == 0
  uint64_t obs_mask;  // Lorenz '96: bit n set iff component n is observed
  uint64_t seed;
  double dt, thr;
  double theta[8];
  void* x[2];         // state double buffer, component-major [N][P]
  double* ctil;       // in-tile inclusive prefix of exp(ell - M_tile) [P]
  double* ell;        // log-weights (adaptive / never modes) [P]
  double* lam;        // carried log-weights [P]
  int32_t* anc;       // ancestors: [P], or [T][P] history when hist != 0
  const double* y;    // observations [T][Ny]
  const double* flow; // windkessel input F(k dt), k = 0..T*s
  TilePart* tp;       // [ntiles]
  GroupPart* gp;      // [ngroups]
  Ctl* ctl;
  double* mn_t;       // multinomial: in-tile inclusive sums of the spacings [P]
  double* mn_part;    // multinomial: tile offsets [ntiles], then P / (sum of all P + 1)
  const double* znoise;  // FP64 windkessel: normals drawn ahead, [T * s][P], or null
};
static_assert(sizeof(FilterDev) == 272, "descriptor layout");

// Work queue of the batched form's persistent launch (k_persist).  Items are
// 64-bit words (filter + 1) << 32 | phase << 24 | q: the tiles
// [q kt, (q + 1) kt) of one filter to propagate (PHASE_PROP), or the tiles
// [q RS_CHUNK, (q + 1) RS_CHUNK) to resample (PHASE_RS), at the filter's
// current step; 0 marks a slot not yet filled.  An item goes to one of
// PERSIST_LEVELS first-in-first-out levels by its filter's remaining phases
// (persist_level: the longest remaining runs first).  Per level, slots are
// filled once per run in order of reservation (tail) and taken in order
// (head); total is the number of items the run puts in the level, lowered
// when a filter ends early (a degenerate step); base is the level's first
// slot in the slot array.
constexpr int PERSIST_LEVELS = 8;
struct alignas(128) PersistLevel {
  unsigned long long head;   // next slot to take
  unsigned long long tail;   // next slot to fill
  unsigned long long total;  // slots the run fills
  unsigned long long base;   // first slot in the slot array
  unsigned long long cap;    // slots allocated
};
struct alignas(128) PersistQueue {
  PersistLevel lv[PERSIST_LEVELS];
  int maxT;                  // the longest listed run (levels scale with it)
  int err;                   // this run: a wait ran out (1), a push overflowed (2), an
                             // item of a stopped filter or a class outside the kernel's (3)
  int err_any;               // every run since the plan was built (not reset per run)
};
// Level of an item whose filter has rem >= 1 phases of its kind left,
// including this one (a propagate item of step i: T - i + 1; a resample
// item of step i: T - i), in a launch whose longest run has maxT steps.
__host__ __device__ constexpr int persist_level(int rem, int maxT) {
  return int((static_cast<long long>(rem) * PERSIST_LEVELS) / (static_cast<long long>(maxT) + 1));
}
enum { PHASE_PROP = 1, PHASE_RS = 2 };
__host__ __device__ constexpr unsigned long long persist_item(int k, int phase, int q) {
  return (static_cast<unsigned long long>(k + 1) << 32) |
         (static_cast<unsigned long long>(phase) << 24) | static_cast<unsigned long long>(q);
}
// Model classes the persistent kernel is compiled for, as bits of its class set.
enum { PC_WK64 = 1, PC_WK32 = 2, PC_L8_64 = 4, PC_L8_32 = 8 };

// -------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
// 32x32->64 multiplies and xors, key bumped by the Weyl increments between
// rounds.
// -------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo_a = 0xD2511F53u * c.x;
    const uint32_t hi_a = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo_b = 0xCD9E8D57u * c.z;
    const uint32_t hi_b = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi_b ^ c.y ^ k0, lo_b, hi_a ^ c.w ^ k1, lo_a);
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

// Block of the stream (particle j, step i, purpose): counter (j, i, purpose<<16 | b, 0).
__device__ __forceinline__ uint4 rng_block(uint64_t seed, uint32_t j, uint32_t i, uint32_t purpose,
                                           uint32_t b) {
  return philox4x32_10(make_uint4(j, i, (purpose << 16) | b, 0u), uint32_t(seed),
                       uint32_t(seed >> 32));
}

// 53-bit uniforms from the 64-bit word hi:lo.
__device__ __forceinline__ double u53_closed_open(uint32_t lo, uint32_t hi) {  // [0,1)
  const unsigned long long v = ((static_cast<unsigned long long>(hi) << 32) | lo) >> 11;
  return __dmul_rn(__ull2double_rn(v), 0x1.0p-53);
}
__device__ __forceinline__ double u53_open_closed(uint32_t lo, uint32_t hi) {  // (0,1]
  const unsigned long long v = ((static_cast<unsigned long long>(hi) << 32) | lo) >> 11;
  return __dmul_rn(__ull2double_rn(v + 1ull), 0x1.0p-53);
}

// -------------------------------------------------------------------------
// Natural logarithm, FP64, for positive normal x: x = m 2^e with m in
// [1/sqrt2, sqrt2) read off the bits, log m = 2 atanh((m-1)/(m+1)) by the
// odd series to the 23rd power, plus e ln 2 with ln 2 in two parts.
// -------------------------------------------------------------------------
__device__ __forceinline__ double log_pos(double x) {
  const long long bits = __double_as_longlong(x);
  int e = int((bits >> 52) & 0x7ff) - 1022;
  double m = __longlong_as_double((bits & 0x000fffffffffffffLL) | 0x3fe0000000000000LL);
  if (m < 0x1.6a09e667f3bcdp-1) {
    m = __dadd_rn(m, m);
    e -= 1;
  }
  const double f = __ddiv_rn(__dsub_rn(m, 1.0), __dadd_rn(m, 1.0));
  const double two_f = __dadd_rn(f, f);
  const double f2 = __dmul_rn(f, f);
  double p = 1.0 / 23.0;
  p = fma(p, f2, 1.0 / 21.0);
  p = fma(p, f2, 1.0 / 19.0);
  p = fma(p, f2, 1.0 / 17.0);
  p = fma(p, f2, 1.0 / 15.0);
  p = fma(p, f2, 1.0 / 13.0);
  p = fma(p, f2, 1.0 / 11.0);
  p = fma(p, f2, 1.0 / 9.0);
  p = fma(p, f2, 1.0 / 7.0);
  p = fma(p, f2, 1.0 / 5.0);
  p = fma(p, f2, 1.0 / 3.0);
  const double lm = fma(__dmul_rn(two_f, f2), p, two_f);
  const double de = double(e);
  return fma(de, 0x1.62e42fefa39efp-1, fma(de, 0x1.abc9e3b39803fp-56, lm));
}

// Exponential, FP64 (Cody and Waite): k = rint(x / ln2), r = x - k ln2 with
// ln2 in two parts, e^r by its Taylor series to r^14, e^x = e^r 2^k; used
// where the state itself depends on an exponential.
__device__ __forceinline__ double exp_own(double x) {
  if (x != x) return x;
  if (x > 709.782712893384) return INFINITY;
  if (x < -745.1332191019412) return 0.0;
  const double k = rint(__dmul_rn(x, 0x1.71547652b82fep+0));
  double r = fma(-k, 0x1.62e42fefa39efp-1, x);
  r = fma(-k, 0x1.abc9e3b39803fp-56, r);
  double p = 1.0 / 87178291200.0;
  p = fma(p, r, 1.0 / 6227020800.0);
  p = fma(p, r, 1.0 / 479001600.0);
  p = fma(p, r, 1.0 / 39916800.0);
  p = fma(p, r, 1.0 / 3628800.0);
  p = fma(p, r, 1.0 / 362880.0);
  p = fma(p, r, 1.0 / 40320.0);
  p = fma(p, r, 1.0 / 5040.0);
  p = fma(p, r, 1.0 / 720.0);
  p = fma(p, r, 1.0 / 120.0);
  p = fma(p, r, 1.0 / 24.0);
  p = fma(p, r, 1.0 / 6.0);
  p = fma(p, r, 0.5);
  p = fma(p, r, 1.0);
  p = fma(p, r, 1.0);
  return ldexp(p, int(k));
}

// sin(2 pi u), cos(2 pi u), FP64, u in [0,1): quarter turns q = rint(4u),
// remainder r = 4u - q (exact), angle r pi/2 with pi/2 in two parts, Taylor
// series of sin to x^19 and cos to x^20, then rotation by q quarter turns.
__device__ __forceinline__ void sincos_2pi(double u, double* sn, double* cs) {
  const double v = __dmul_rn(4.0, u);
  const double q = rint(v);
  const double r = __dsub_rn(v, q);
  const double x = fma(r, 0x1.921fb54442d18p+0, __dmul_rn(r, 0x1.1a62633145c07p-54));
  const double x2 = __dmul_rn(x, x);
  double s = -1.0 / 121645100408832000.0;
  s = fma(s, x2, 1.0 / 355687428096000.0);
  s = fma(s, x2, -1.0 / 1307674368000.0);
  s = fma(s, x2, 1.0 / 6227020800.0);
  s = fma(s, x2, -1.0 / 39916800.0);
  s = fma(s, x2, 1.0 / 362880.0);
  s = fma(s, x2, -1.0 / 5040.0);
  s = fma(s, x2, 1.0 / 120.0);
  s = fma(s, x2, -1.0 / 6.0);
  const double sinx = fma(__dmul_rn(x, x2), s, x);
  double c = 1.0 / 2432902008176640000.0;
  c = fma(c, x2, -1.0 / 6402373705728000.0);
  c = fma(c, x2, 1.0 / 20922789888000.0);
  c = fma(c, x2, -1.0 / 87178291200.0);
  c = fma(c, x2, 1.0 / 479001600.0);
  c = fma(c, x2, -1.0 / 3628800.0);
  c = fma(c, x2, 1.0 / 40320.0);
  c = fma(c, x2, -1.0 / 720.0);
  c = fma(c, x2, 1.0 / 24.0);
  c = fma(c, x2, -0.5);
  const double cosx = fma(x2, c, 1.0);
  const int quarter = int(q) & 3;
  *sn = quarter == 0 ? sinx : quarter == 1 ? cosx : quarter == 2 ? -sinx : -cosx;
  *cs = quarter == 0 ? cosx : quarter == 1 ? -sinx : quarter == 2 ? -cosx : sinx;
}

// FP32 versions of the same two methods, series cut for single precision.
__device__ __forceinline__ float log_posf(float x) {
  const int bits = __float_as_int(x);
  int e = ((bits >> 23) & 0xff) - 126;
  float m = __int_as_float((bits & 0x007fffff) | 0x3f000000);
  if (m < 0x1.6a09e6p-1f) {
    m = __fadd_rn(m, m);
    e -= 1;
  }
  const float f = __fdiv_rn(__fsub_rn(m, 1.0f), __fadd_rn(m, 1.0f));
  const float two_f = __fadd_rn(f, f);
  const float f2 = __fmul_rn(f, f);
  float p = 1.0f / 11.0f;
  p = fmaf(p, f2, 1.0f / 9.0f);
  p = fmaf(p, f2, 1.0f / 7.0f);
  p = fmaf(p, f2, 1.0f / 5.0f);
  p = fmaf(p, f2, 1.0f / 3.0f);
  const float lm = fmaf(__fmul_rn(two_f, f2), p, two_f);
  const float de = float(e);
  return fmaf(de, 0x1.62e430p-1f, fmaf(de, -0x1.05c610p-29f, lm));
}

__device__ __forceinline__ void sincos_2pif(float u, float* sn, float* cs) {
  const float v = __fmul_rn(4.0f, u);
  const float q = rintf(v);
  const float r = __fsub_rn(v, q);
  const float x = fmaf(r, 0x1.921fb6p+0f, __fmul_rn(r, -0x1.777a5cp-25f));
  const float x2 = __fmul_rn(x, x);
  float s = -1.0f / 39916800.0f;
  s = fmaf(s, x2, 1.0f / 362880.0f);
  s = fmaf(s, x2, -1.0f / 5040.0f);
  s = fmaf(s, x2, 1.0f / 120.0f);
  s = fmaf(s, x2, -1.0f / 6.0f);
  const float sinx = fmaf(__fmul_rn(x, x2), s, x);
  float c = 1.0f / 479001600.0f;
  c = fmaf(c, x2, -1.0f / 3628800.0f);
  c = fmaf(c, x2, 1.0f / 40320.0f);
  c = fmaf(c, x2, -1.0f / 720.0f);
  c = fmaf(c, x2, 1.0f / 24.0f);
  c = fmaf(c, x2, -0.5f);
  const float cosx = fmaf(x2, c, 1.0f);
  const int quarter = int(q) & 3;
  *sn = quarter == 0 ? sinx : quarter == 1 ? cosx : quarter == 2 ? -sinx : -cosx;
  *cs = quarter == 0 ? cosx : quarter == 1 ? -sinx : quarter == 2 ? -cosx : sinx;
}

// Box-Muller pair from one Philox block (FP64): u1 in (0,1] from w1:w0,
// u2 in [0,1) from w3:w2; z0 = rho cos, z1 = rho sin.
__device__ __forceinline__ void normal_pair64(uint4 w, double* z0, double* z1) {
  const double u1 = u53_open_closed(w.x, w.y);
  const double u2 = u53_closed_open(w.z, w.w);
  const double rho = __dsqrt_rn(__dmul_rn(-2.0, log_pos(u1)));
  double sn, cs;
  sincos_2pi(u2, &sn, &cs);
  *z0 = __dmul_rn(rho, cs);
  *z1 = __dmul_rn(rho, sn);
}

// ---------------------------------------------------------------------------
// Packed FP32 pairs (sm_100-family f32x2 instructions): one instruction does
// the same IEEE single-precision operation on both halves of a 64-bit
// register, so a packed computation gives bit for bit the scalar results
// with half the instructions issued.
// ---------------------------------------------------------------------------
typedef unsigned long long f32x2;

__device__ __forceinline__ f32x2 pk(float lo, float hi) {
  f32x2 d;
  asm("mov.b64 %0, {%1, %2};" : "=l"(d) : "f"(lo), "f"(hi));
  return d;
}
__device__ __forceinline__ void upk(f32x2 v, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f32x2 swp(f32x2 v) {
  float a, b;
  upk(v, a, b);
  return pk(b, a);
}
__device__ __forceinline__ f32x2 fma2(f32x2 a, f32x2 b, f32x2 c) {
  f32x2 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ f32x2 sub2(f32x2 a, f32x2 b) {
  f32x2 d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}

// FP32: one 32-bit word pair (a, b) gives one pair: u1 = ((a>>8)+1) 2^-24,
// u2 = (b>>8) 2^-24.
__device__ __forceinline__ void normal_pair32(uint32_t a, uint32_t b, float* z0, float* z1) {
  const float u1 = __fmul_rn(float((a >> 8) + 1u), 0x1.0p-24f);
  const float u2 = __fmul_rn(float(b >> 8), 0x1.0p-24f);
  const float rho = __fsqrt_rn(__fmul_rn(-2.0f, log_posf(u1)));
  float sn, cs;
  sincos_2pif(u2, &sn, &cs);
  *z0 = __fmul_rn(rho, cs);
  *z1 = __fmul_rn(rho, sn);
}

// -------------------------------------------------------------------------
// Order-preserving int64 key of a double (for max by integer compare).
// -------------------------------------------------------------------------
__device__ __forceinline__ long long dkey(double v) {
  const long long b = __double_as_longlong(v);
  return b ^ ((b >> 63) & 0x7fffffffffffffffLL);
}
__device__ __forceinline__ double dunkey(long long k) {
  return __longlong_as_double(k ^ ((k >> 63) & 0x7fffffffffffffffLL));
}

// Scratch for the canonical block operations (TILE threads).
struct BlockScratch {
  long long kmax[WARPS];
  unsigned long long usum[WARPS];  // block_scan_fixed: the warps' totals
  double wsum[WARPS];
  double wsum2[WARPS];
  double wpre[WARPS];
  double wtot;
  int flag;
};

// Max over the block; every thread receives it.
__device__ __forceinline__ double block_max(double v, BlockScratch& sm) {
  long long k = dkey(v);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) k = max(k, __shfl_xor_sync(0xffffffffu, k, o));
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) sm.kmax[w] = k;
  __syncthreads();
  long long r = sm.kmax[0];
#pragma unroll
  for (int q = 1; q < WARPS; ++q) r = max(r, sm.kmax[q]);
  __syncthreads();
  return dunkey(r);
}

// Canonical sum: xor-butterfly inside each warp, then the eight warp totals
// combined as ((w0+w1)+(w2+w3))+((w4+w5)+(w6+w7)).  Every thread receives it.
__device__ __forceinline__ double block_sum(double v, BlockScratch& sm) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = __dadd_rn(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) sm.wsum2[w] = v;
  __syncthreads();
  const double* t = sm.wsum2;
  const double r = __dadd_rn(__dadd_rn(__dadd_rn(t[0], t[1]), __dadd_rn(t[2], t[3])),
                             __dadd_rn(__dadd_rn(t[4], t[5]), __dadd_rn(t[6], t[7])));
  __syncthreads();
  return r;
}

// Canonical inclusive scan: Kogge-Stone inside each warp (shfl_up 1..16),
// then warp 0 scans the eight warp totals with a Kogge-Stone over lanes 0..7
// (shfl_up 1, 2, 4) and every thread adds its warp's exclusive prefix.
// Returns the thread's inclusive prefix; *total receives the block total.
__device__ __forceinline__ double block_scan(double v, BlockScratch& sm, double* total) {
  const int lane = threadIdx.x & 31;
  const int w = threadIdx.x >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const double n = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v = __dadd_rn(n, v);
  }
  if (lane == 31) sm.wsum[w] = v;
  __syncthreads();
  if (w == 0) {
    double t = lane < WARPS ? sm.wsum[lane] : 0.0;
#pragma unroll
    for (int o = 1; o < WARPS; o <<= 1) {
      const double n = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t = __dadd_rn(n, t);
    }
    const double ex = __shfl_up_sync(0xffffffffu, t, 1);
    if (lane < WARPS) sm.wpre[lane] = lane == 0 ? 0.0 : ex;
    if (lane == WARPS - 1) sm.wtot = t;
  }
  __syncthreads();
  *total = sm.wtot;
  return w == 0 ? v : __dadd_rn(sm.wpre[w], v);
}

// ---------------------------------------------------------------------------
// The in-tile cumulative weights, exactly.  A weight w = exp(ell - M_t) lies
// in [0, 1], so w 2^55 rounded to an integer (weight_fixed) and the sum of a
// tile's 256 of them (at most 2^63) are exact unsigned 64-bit integers: the
// scan (block_scan_fixed) has no rounding and no order, and each prefix is
// rounded once to the nearest double (fixed_double).  The resolution, 2^-55
// of the tile's largest weight, is finer than a double's at the tile total
// (>= 1); all of it is integer work, none on the FP64 unit (B300: 1/64 of the
// FP32 rate).
// ---------------------------------------------------------------------------
// round(w 2^55) for 0 <= w <= 1, read off the IEEE-754 fields: w = m 2^(e-52)
// with the 53-bit significand m (no hidden bit for a subnormal), so
// w 2^55 = m 2^(e+3): a left shift of at most 3 (w <= 1), or a right shift
// rounded to nearest, ties to even.
__device__ __forceinline__ unsigned long long weight_fixed(double w) {
  const unsigned long long b =
      static_cast<unsigned long long>(__double_as_longlong(w)) & 0x7fffffffffffffffull;  // -0: 0
  const int E = int(b >> 52);  // biased exponent
  const unsigned long long m = (b & 0x000fffffffffffffull) | (E ? 0x0010000000000000ull : 0ull);
  const int sh = (E ? E : 1) - 1023 + 3;
  if (sh >= 0) return m << sh;
  const int r = -sh;
  if (r > 54) return 0ull;  // m 2^-r < 1/2
  const unsigned long long q = m >> r;
  const unsigned long long rem = m & ((1ull << r) - 1ull);
  const unsigned long long half = 1ull << (r - 1);
  return q + ((rem > half || (rem == half && (q & 1ull))) ? 1ull : 0ull);
}

// p 2^-55 rounded to the nearest double (ties to even), for p < 2^64: the
// leading bit of p sets the exponent; the result is 0 or a normal number.
__device__ __forceinline__ double fixed_double(unsigned long long p) {
  if (p == 0ull) return 0.0;
  const int top = 63 - __clzll(static_cast<long long>(p));  // leading bit of p
  int e = top - 55;  // unbiased exponent of p 2^-55
  unsigned long long m;
  if (top <= 52) {
    m = p << (52 - top);
  } else {
    const int r = top - 52;
    const unsigned long long q = p >> r;
    const unsigned long long rem = p & ((1ull << r) - 1ull);
    const unsigned long long half = 1ull << (r - 1);
    m = q + ((rem > half || (rem == half && (q & 1ull))) ? 1ull : 0ull);
    if (m == (1ull << 53)) {
      m >>= 1;
      e += 1;
    }
  }
  return __longlong_as_double(static_cast<long long>(
      (static_cast<unsigned long long>(e + 1023) << 52) | (m & 0x000fffffffffffffull)));
}

// Inclusive scan of v over the block, exact in unsigned 64-bit integers: a
// shuffle scan in each warp, then every thread adds the totals of the warps
// before its own (one barrier).  total receives the block's sum.
__device__ __forceinline__ unsigned long long block_scan_fixed(unsigned long long v,
                                                               BlockScratch& sm,
                                                               unsigned long long* total) {
  const int lane = threadIdx.x & 31;
  const int w = threadIdx.x >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long n = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += n;
  }
  if (lane == 31) sm.usum[w] = v;
  __syncthreads();
  unsigned long long before = 0ull, all = 0ull;
#pragma unroll
  for (int q = 0; q < WARPS; ++q) {
    const unsigned long long t = sm.usum[q];
    if (q < w) before += t;
    all += t;
  }
  *total = all;
  return v + before;
}

// Warp-level forms of the three canonical reductions for inputs held by the
// lanes of one warp, the other warps' inputs being the neutral element (0 for
// sums and scans, -inf for the max): block_max, block_sum and block_scan then
// reduce the seven other warp totals to the neutral element, and x + 0 = x, so
// these give the same bits with no block barrier.
__device__ __forceinline__ double warp_max(double v) {
  long long k = dkey(v);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) k = max(k, __shfl_xor_sync(0xffffffffu, k, o));
  return dunkey(k);
}
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = __dadd_rn(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ double warp_scan(double v, double* total) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const double n = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v = __dadd_rn(n, v);
  }
  *total = __shfl_sync(0xffffffffu, v, 31);
  return v;
}

// L2-coherent loads for data written by other blocks of the same launch.
template <typename T>
__device__ __forceinline__ T ldcg(const T* p) {
  return __ldcg(p);
}

}  // namespace pfb
