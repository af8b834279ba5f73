// Device-side definitions shared by the CUDA translation units of libtpcg.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "tpcg_internal.h"

namespace tpcg {

// Scalars of one PCG solve (Algorithm 1), kept in device memory so that the
// iteration runs without host round trips.  Written only by the last block
// of a reduction ("finalize"), read by every later kernel.
// Mixed forms: the directions P_k kept in a ring for the deferred update of U (k_form_u).
constexpr int kPRing = 8;

struct SolveState {
  double mean_eta;     // mean removed from eta (eq. centering) when singular
  double eta_norm2;    // ||eta_hat||^2
  double tol2;         // tol^2 * ||eta_hat||^2
  double rr;           // ||R_s||^2 of the recurrence
  double sumR;         // sum(R_s)
  double rho;          // rho_s = <R_s, Z_s'> with Z' the centred Z
  double beta;         // beta_s
  double alpha;        // alpha_s
  double mZ;           // mean of Z_s (centring, Remark orthogonality)
  double pWp;          // <W_s, P_{s-1}>
  double nah[3];       // -alpha_s / h^2 per axis (set with alpha)
  double true_rr;      // ||eta_hat - L U||^2 at the last FP64 check
  double sumU;         // sum(U) at the last FP64 check
  double zscale;       // power-of-two scale applied to R before low-precision conversion
  const double* eta;   // the solve's right-hand side and iterate (device pointers): the kernels that touch
  double* ups;         // them read them here, so one captured launch sequence serves every solve of a plan
  int iter;            // s
  int maxit;
  int done;            // 1: stop issuing work
  int status;          // TPCG_* code
  int need_check;      // recurrence says converged (or maxit): evaluate the true residual
  int first;           // 1 until the first direction P_0 = Z_0' has been formed
  int zero_guess;      // U_0 = 0: the first update writes U instead of adding
  int singular;
  int precond_applies;
  int checks;          // true-residual evaluations
  int done_iter;       // iteration whose true-residual check met the tolerance (0: none)
  int timeout;         // a bounded device wait gave up
  unsigned zmax_bits;  // max |Z| accumulator of the preconditioner output (FP32 bits; atomicMax)
  float zmax;          // max |Z| of the current preconditioner output
  int kp;              // mixed forms: P_s = P_int * 2^-kp, |P_int| <= 2^20 (exact fixed point)
  int kp_next;         // exponent of the next direction (set with beta by the preconditioner finalize)
  float bs_next;       // beta * 2^-kp (FP32) for the next direction
  unsigned pmax_bits;  // max |P_int| accumulator of the direction kernel (atomicMax)
  double pmax;         // max |P_s| of the current direction
  unsigned long long umax_bits;  // max |U| accumulator (FP64 bits of |U|; atomicMax)
  double umax;         // max |U| of the current iterate
  int ku;              // fixed-point exponent of U for the residual check (from umax)
  int sr;              // 2^-sr bounds every |eta_hat - L U| entry (scale of the check's FP32 sums)
  int lp_shift;        // power-of-two exponent applied when R is next converted to FP16
  int lp_shift_applied;  // exponent the current low-precision copy of R was converted with
  unsigned tickets[8]; // arrival counters of the last-block reductions
  // mixed forms, deferred U += alpha_k P_k (k_form_u): alpha_k, the exponent of P_k and its ring slot
  int n_pend;          // updates recorded and not yet applied to U
  int u_valid;         // U holds an iterate (0: zero initial guess and no update applied yet)
  double pend_alpha[kPRing];
  int pend_kp[kPRing];
  int pend_slot[kPRing];
};

enum Ticket { kTkEta = 0, kTkInit = 1, kTkDir = 2, kTkUpd = 3, kTkTrue = 4, kTkPrec = 5, kTkMisc = 6, kTkForm = 7 };

// Geometry of a grid and its stencil (eq. lap1d / eq. ourproblem).
struct Geom {
  int nx, ny, nz;
  int bc[3];
  double ih2[3];   // 1/h^2 per axis (0 for an absent z axis)
  float ih2f[3];   // the same in FP32, converted on the host: FP64 -> FP32
                   // conversions issue on the slow FP64 pipe of this part
  double nih2[3];  // -1/h^2 per axis
  int uniform;     // all present axes share one spacing
  long long N;     // nx*ny*nz
};

// Counts a kernel launch of the plan and, when profiling is on, brackets it
// with CUDA events on the plan's stream.
struct LaunchScope {
  const tpcg_plan* p;
  int kind;
  cudaEvent_t b = nullptr;
  LaunchScope(const tpcg_plan* plan, int k) : p(plan), kind(k) {
    p->launch_count += 1;
    p->prof.launches[k] += 1;
    if (p->prof.on) {
      cudaEvent_t a = take_event(), e = take_event();
      if (a && e) {
        cudaEventRecord(a, p->stream);
        b = e;
        p->prof.recs.push_back({k, {a, e}});
      }
    }
  }
  ~LaunchScope() {
    if (b) cudaEventRecord(b, p->stream);
  }
  cudaEvent_t take_event() {
    Profiler& pr = p->prof;
    if (pr.used < pr.pool.size()) return pr.pool[pr.used++];
    cudaEvent_t ev = nullptr;
    if (cudaEventCreate(&ev) != cudaSuccess) return nullptr;
    pr.pool.push_back(ev);
    pr.used = pr.pool.size();
    return ev;
  }
};

// Block-wide sum of NQ doubles; result valid in thread 0.  Fixed order: the
// result is bitwise reproducible for a fixed launch configuration.
template <int NQ>
__device__ __forceinline__ void block_sum(double (&v)[NQ], double* sh /* NQ*32 doubles */) {
  const int lane = threadIdx.x & 31;
  const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  const int warp = tid >> 5;
  const int nthreads = blockDim.x * blockDim.y * blockDim.z;
  const int nwarps = (nthreads + 31) >> 5;
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    double x = v[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if (lane == 0) sh[q * 32 + warp] = x;
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      double x = (lane < nwarps) ? sh[q * 32 + lane] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
      v[q] = x;
    }
  }
  __syncthreads();
}

// Deterministic grid-wide reduction: every block stores its partial sums,
// the last block to arrive adds all partials in block order and calls
// fin(sums) from thread 0.  Returns true in the finishing thread.
template <int NQ, class Fin>
__device__ __forceinline__ void grid_reduce(double (&v)[NQ], double* partials, unsigned* ticket, int nblocks,
                                            int block_id, Fin fin) {
  __shared__ double sh[NQ * 32];
  __shared__ bool last;
  block_sum<NQ>(v, sh);
  const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  const int nthreads = blockDim.x * blockDim.y * blockDim.z;
  if (tid == 0) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) partials[(size_t)block_id * NQ + q] = v[q];
    __threadfence();
    unsigned t = atomicAdd(ticket, 1u);
    last = (t == (unsigned)nblocks - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double s[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) s[q] = 0.0;
  for (int b = tid; b < nblocks; b += nthreads) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) s[q] += __ldcg(&partials[(size_t)b * NQ + q]);
  }
  block_sum<NQ>(s, sh);
  if (tid == 0) {
    fin(s);
    *ticket = 0u;
  }
}

// Finalize of one preconditioner application inside PCG (Algorithm 1):
// centre Z (Remark orthogonality), rho_s = <R_s, Z_s - mean Z_s>, beta_s.
__device__ __forceinline__ void fin_precond(SolveState* st, long long N, const double (&s)[2]) {
  const double mZ = st->singular ? s[1] / (double)N : 0.0;
  const double rho = s[0] - mZ * st->sumR;
  st->mZ = mZ;
  st->precond_applies += 1;
  if (!isfinite(rho) || !(rho > 0.0)) {
    if (st->rr == 0.0) {  // exact solution already reached
      st->status = TPCG_OK;
      st->done = 1;
    } else {
      st->status = TPCG_ERR_BREAKDOWN;
      st->done = 1;
    }
    return;
  }
  st->beta = st->first ? 0.0 : rho / st->rho;
  st->rho = rho;
}

// FP64 -> BF16 with round-to-nearest-even done in integer arithmetic on the
// bit pattern (the FP64 conversion pipe is slow on this part).  Values below
// the BF16 normal range flush to signed zero; values above it saturate to the
// largest finite BF16; NaN stays NaN.
__device__ __forceinline__ uint16_t f64_to_bf16_bits(double x) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const uint32_t hi = (uint32_t)(u >> 32);
  const uint32_t sign = (hi >> 16) & 0x8000u;
  const int e = (int)((hi >> 20) & 0x7ff);
  if (e == 0x7ff) return (uint16_t)(sign | 0x7f80u | (((u & 0xfffffffffffffull) != 0) ? 0x40u : 0u));
  const int eb = e - 1023 + 127;             // BF16 biased exponent
  if (eb <= 0) return (uint16_t)sign;        // underflow: signed zero
  const unsigned long long mant = u & 0xfffffffffffffull;  // 52 bits
  uint32_t top = (uint32_t)(mant >> 45);     // 7 kept bits
  const unsigned long long rest = mant & ((1ull << 45) - 1);
  const unsigned long long halfway = 1ull << 44;
  uint32_t bits = ((uint32_t)eb << 7) | top;
  if (rest > halfway || (rest == halfway && (top & 1u))) bits += 1;  // carry may bump exponent: correct
  if (bits >= 0x7f80u) bits = 0x7f7fu;       // saturate
  return (uint16_t)(sign | bits);
}

// x * 2^shift -> FP32 with round-to-nearest-even in integer arithmetic;
// underflow to signed zero below the FP32 normal range, saturation above.
__device__ __forceinline__ float f64_to_f32_int(double x, int shift = 0) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const uint32_t sign = (uint32_t)(u >> 32) & 0x80000000u;
  const int e = (int)((u >> 52) & 0x7ff);
  if (e == 0x7ff) return __uint_as_float(sign | 0x7f800000u | (((u & 0xfffffffffffffull) != 0) ? 0x400000u : 0u));
  if (e == 0) return __uint_as_float(sign);
  const int eb = e - 1023 + 127 + shift;
  if (eb <= 0) return __uint_as_float(sign);
  const unsigned long long mant = u & 0xfffffffffffffull;
  uint32_t top = (uint32_t)(mant >> 29);     // 23 kept bits
  const uint32_t rest = (uint32_t)(mant & ((1u << 29) - 1));
  const uint32_t halfway = 1u << 28;
  uint32_t bits = ((uint32_t)eb << 23) | top;
  if (rest > halfway || (rest == halfway && (top & 1u))) bits += 1;
  if (bits >= 0x7f800000u) bits = 0x7f7fffffu;
  return __uint_as_float(sign | bits);
}

// x * 2^shift -> FP16 (binary16), round-to-nearest-even in integer arithmetic,
// gradual underflow to FP16 subnormals, saturation to the largest finite
// value (65504) above the range; NaN/Inf pass through.
__device__ __forceinline__ uint16_t f64_to_f16_bits(double x, int shift) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const uint32_t sign = (uint32_t)(u >> 48) & 0x8000u;
  const int e = (int)((u >> 52) & 0x7ff);
  if (e == 0x7ff) return (uint16_t)(sign | 0x7c00u | (((u & 0xfffffffffffffull) != 0) ? 0x200u : 0u));
  if (e == 0) return (uint16_t)sign;
  const int E = e - 1023 + shift;
  if (E > 15) return (uint16_t)(sign | 0x7bffu);
  const unsigned long long m = (u & 0xfffffffffffffull) | (1ull << 52);
  int sh = 42;
  uint32_t ef = 0;
  if (E >= -14) {
    ef = (uint32_t)(E + 15);
  } else {
    sh = 28 - E;
    if (sh > 62) return (uint16_t)sign;
  }
  const unsigned long long qv = m >> sh;
  const unsigned long long rem = m & ((1ull << sh) - 1);
  const unsigned long long half = 1ull << (sh - 1);
  uint32_t bits = ef ? ((ef << 10) | ((uint32_t)qv & 0x3ffu)) : (uint32_t)qv;
  if (rem > half || (rem == half && (qv & 1ull))) bits += 1;
  if (bits >= 0x7c00u) bits = 0x7bffu;
  return (uint16_t)(sign | bits);
}

// Exponent s with rms * 2^s in [0.5, 1) for the FP16 copy of a vector of
// squared 2-norm n2 and length N (0 when the vector is zero).
__device__ __forceinline__ int lp_shift_for(double n2, long long N) {
  if (!(n2 > 0.0) || !isfinite(n2)) return 0;
  const double rms = sqrt(n2 / (double)N);
  int s = -ilogb(rms) - 1;
  return s < -120 ? -120 : (s > 120 ? 120 : s);
}

// round(z * 2^k) as int32 for |z * 2^k| < 2^30 (round-to-nearest-even, integer
// arithmetic on the bit pattern).  FP32 subnormals map to 0.
__device__ __forceinline__ int f32_to_fixed(float z, int k) {
  const uint32_t b = __float_as_uint(z);
  const int e = (int)((b >> 23) & 0xff);
  if (e == 0) return 0;
  const uint32_t m = (b & 0x7fffffu) | 0x800000u;
  const int sh = e - 150 + k;  // z * 2^k = m * 2^sh
  uint32_t q;
  if (sh >= 0) {
    q = m << sh;
  } else if (sh < -25) {
    q = 0;
  } else {
    q = m >> -sh;
    const uint32_t rem = m & ((1u << -sh) - 1u), half = 1u << (-sh - 1);
    if (rem > half || (rem == half && (q & 1u))) ++q;
  }
  return (b >> 31) ? -(int)q : (int)q;
}

// v * 2^e as FP64 for |v| < 2^31 (exact), built on the bit pattern: the
// leading one of the shifted magnitude lands on bit 52 and is added into the
// exponent field, which is therefore written one lower.
__device__ __forceinline__ double i32_to_f64_scaled(int v, int e) {
  if (v == 0) return 0.0;
  const uint32_t a = v < 0 ? 0u - (uint32_t)v : (uint32_t)v;
  const int msb = 31 - __clz(a);
  const unsigned long long bits = ((unsigned long long)(uint32_t)(v < 0) << 63) +
                                  ((unsigned long long)(msb + e + 1022) << 52) +
                                  ((unsigned long long)a << (52 - msb));
  return __longlong_as_double((long long)bits);
}

// Exponent k with bound * 2^k < 2^20 for the fixed-point direction
// (bound >= max|P|); 0 when the bound is zero.  With |P_int| <= 2^20 every
// difference of two values is below 2^22 and converts to FP32 exactly by the
// magic-number rule below, and every 7-point stencil fits in 24 bits.
__device__ __forceinline__ int fixed_shift_for(double bound) {
  if (!(bound > 0.0) || !isfinite(bound)) return 0;
  const int k = 19 - ilogb(bound);
  return k < -900 ? -900 : (k > 900 ? 900 : k);
}

// Exact int -> FP32 for |v| < 2^22 without a conversion instruction (those
// issue on the slow FP64 pipe of this part): 1.5 * 2^23 + v is exact in FP32.
__device__ __forceinline__ float i22_to_f32(int v) { return __int_as_float(0x4B400000 + v) - 12582912.0f; }

// round(v * sc) as int for |v * sc| < 2^22, round-to-nearest-even: one FMA
// against 1.5 * 2^23, whose ulp is 1.
__device__ __forceinline__ int f32_to_i22(float v, float sc) {
  return __float_as_int(fmaf(v, sc, 12582912.0f)) - 0x4B400000;
}

// x * 2^shift -> FP32 with round-to-odd (truncate, then set the last bit when
// anything was cut off), on the bit pattern.  Rounding this value to FP16 or
// BF16 with round-to-nearest-even gives exactly the correctly rounded x * 2^shift
// (round-to-odd keeps the sticky information; FP32 has more than two extra
// bits over either target).  Below the FP32 normal range: signed zero; above:
// the largest finite FP32.
__device__ __forceinline__ float f64_to_f32_odd(double x, int shift) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const uint32_t sign = (uint32_t)(u >> 32) & 0x80000000u;
  const int e = (int)((u >> 52) & 0x7ff);
  const int eb = e - 1023 + 127 + shift;
  if (e == 0 || eb <= 0) return __uint_as_float(sign);
  if (e == 0x7ff) return __uint_as_float(sign | 0x7f800000u | (((u & 0xfffffffffffffull) != 0) ? 0x400000u : 0u));
  if (eb >= 255) return __uint_as_float(sign | 0x7f7fffffu);
  const uint32_t top = (uint32_t)(u >> 29) & 0x7fffffu;
  const uint32_t sticky = ((uint32_t)u & ((1u << 29) - 1u)) != 0u;
  return __uint_as_float(sign | ((uint32_t)eb << 23) | top | sticky);
}

// FP32 -> FP16 / BF16 bits, round-to-nearest-even, through the packed
// conversion (which does not issue on the FP64 pipe).
__device__ __forceinline__ uint16_t f32_to_f16_bits_rn(float v) {
  const __half2 h = __floats2half2_rn(v, v);
  return (uint16_t)(*reinterpret_cast<const uint32_t*>(&h) & 0xffffu);
}
__device__ __forceinline__ uint16_t f32_to_bf16_bits_rn(float v) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(v, v);
  return (uint16_t)(*reinterpret_cast<const uint32_t*>(&h) & 0xffffu);
}

// Exponent k with umax * 2^k < 2^58 for the int64 fixed-point residual check:
// twelve such values still sum inside int64.  The clamp keeps every scaled
// result an FP64 normal number.
__device__ __forceinline__ int fixed64_shift_for(double umax) {
  if (!(umax > 0.0) || !isfinite(umax)) return 0;
  const int k = 57 - ilogb(umax);
  return k < -960 ? -960 : (k > 960 ? 960 : k);
}

// round(x * 2^k) as int64 (round-to-nearest-even on the bit pattern) for
// finite x with |x * 2^k| < 2^62; zeros and subnormals give 0.
__device__ __forceinline__ long long f64_to_fixed64(double x, int k) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((u >> 52) & 0x7ff);
  if (e == 0) return 0;
  const unsigned long long m = (u & 0xfffffffffffffull) | (1ull << 52);
  const int sh = e - 1075 + k;  // x * 2^k = m * 2^sh
  unsigned long long q;
  if (sh >= 0) {
    q = m << sh;
  } else if (sh < -54) {
    q = 0;
  } else {
    const int rs = -sh;
    q = m >> rs;
    const unsigned long long rem = m & ((1ull << rs) - 1ull), half = 1ull << (rs - 1);
    if (rem > half || (rem == half && (q & 1ull))) ++q;
  }
  return (u >> 63) ? -(long long)q : (long long)q;
}

// v * 2^e as FP64 with one round-to-nearest-even step, for |v| < 2^63 and a
// result inside the FP64 normal range; built on the bit pattern.
__device__ __forceinline__ double i64_to_f64_scaled(long long v, int e) {
  if (v == 0) return 0.0;
  const unsigned long long sign = v < 0 ? 0x8000000000000000ull : 0ull;
  const unsigned long long a = v < 0 ? 0ull - (unsigned long long)v : (unsigned long long)v;
  const int msb = 63 - __clzll((long long)a);
  unsigned long long mant;
  if (msb <= 52) {
    mant = a << (52 - msb);
  } else {
    const int rs = msb - 52;
    mant = a >> rs;
    const unsigned long long rem = a & ((1ull << rs) - 1ull), half = 1ull << (rs - 1);
    if (rem > half || (rem == half && (mant & 1ull))) ++mant;  // 2^53 carries into the exponent below
  }
  const unsigned long long bits = sign | (((unsigned long long)(msb + e + 1023) << 52) + (mant - (1ull << 52)));
  return __longlong_as_double((long long)bits);
}

// The same value as i64_to_f64_scaled (one round-to-nearest-even step, then an
// exact scaling by 2^e), with the hardware conversion: one operation on the
// FP64 pipe instead of some thirty integer instructions, for kernels with
// FP64-pipe headroom and an instruction-issue bound.  e is added to the
// exponent field, so v * 2^e must be an FP64 normal number (or v == 0).
__device__ __forceinline__ double i64_to_f64_scaled_hw(long long v, int e) {
  const double x = __ll2double_rn(v);
  return v ? __hiloint2double(__double2hiint(x) + (int)((unsigned)e << 20), __double2loint(x)) : 0.0;
}

// FP32 sum with Neumaier's compensation (the rounding error of every addition
// is kept in c); the per-thread partial sums of the PCG scalars use it.
struct Acc32 {
  float s = 0.0f, c = 0.0f;
  __device__ __forceinline__ void add(float x) {
    const float t = s + x;
    c += (fabsf(s) >= fabsf(x)) ? ((s - t) + x) : ((x - t) + s);
    s = t;
  }
};

// FP32 -> FP64 is exact; done on the bit pattern as well.
__device__ __forceinline__ double f32_to_f64_int(float f) {
  const uint32_t b = __float_as_uint(f);
  const uint32_t sign = b & 0x80000000u;
  const uint32_t e = (b >> 23) & 0xff;
  const uint32_t m = b & 0x7fffffu;
  if (e == 0) {
    if (m == 0) return __longlong_as_double((long long)((unsigned long long)sign << 32));
    return (double)f;  // subnormal input: rare, hardware path
  }
  if (e == 0xff) return (double)f;
  const unsigned long long bits = ((unsigned long long)sign << 32) | ((unsigned long long)(e - 127 + 1023) << 52) |
                                  ((unsigned long long)m << 29);
  return __longlong_as_double((long long)bits);
}

// Exponent and beta factor of the next fixed-point direction of the mixed
// forms, from the bound max|Z_s| + |beta_s| max|P_{s-1}| on max|P_s|; called
// once by the preconditioner's finalize, after beta_s is known.
__device__ __forceinline__ void plan_next_direction(SolveState* st) {
  const double bound = (double)st->zmax + (st->first ? 0.0 : fabs(st->beta) * st->pmax);
  st->kp_next = fixed_shift_for(bound);
  st->bs_next = st->first ? 0.0f : (float)ldexp(st->beta, -st->kp);
}

// Scales of the next fixed-point residual check, from max|U| and ||eta_hat||:
// |eta_hat - L U| <= ||eta_hat|| + 12 max(1/h^2) max|U| entrywise.  Set by
// the finalize that last changed U (or measured U_0), read by the check.
__device__ __forceinline__ void plan_residual_check(SolveState* st, const Geom& g) {
  const double umax = st->umax;
  st->ku = fixed64_shift_for(umax);
  const double ihmax = fmax(g.ih2[0], fmax(g.ih2[1], g.ih2[2]));
  const double bound = 2.0 * (sqrt(fmax(st->eta_norm2, 0.0)) + 12.0 * ihmax * umax);
  st->sr = (bound > 0.0 && isfinite(bound)) ? -ilogb(bound) : 0;
}

// Value of a compensated FP32 sum in FP64.
__device__ __forceinline__ double acc_value(const Acc32& a) { return f32_to_f64_int(a.s) + f32_to_f64_int(a.c); }

// Block-wide maximum of an unsigned 64-bit value; result valid in thread 0.
__device__ __forceinline__ unsigned long long block_max_u64(unsigned long long v) {
  __shared__ unsigned long long sh[32];
  const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  const int nthreads = blockDim.x * blockDim.y * blockDim.z;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w > v ? w : v;
  }
  if ((tid & 31) == 0) sh[tid >> 5] = v;
  __syncthreads();
  if (tid == 0) {
    for (int w = 1; w < (nthreads + 31) / 32; ++w) v = sh[w] > v ? sh[w] : v;
  }
  __syncthreads();
  return v;
}

}  // namespace tpcg
