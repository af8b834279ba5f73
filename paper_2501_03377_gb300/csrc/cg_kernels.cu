// FP64 kernels of the PCG iteration (Algorithm 1, Sec. 4.1) around the
// preconditioner: the matrix-free Kronecker-sum stencil of eq. (ourproblem),
// the fused direction / update / residual kernels, centring (eq. centering),
// and the deterministic reductions that produce alpha, beta and the stop test
// on the device.
//
// Stencil scheme: a block owns a 32 x 8 tile of (x, y) columns and marches
// along z through a chunk of planes.  Each plane of the field, with a one-point
// halo in x and y, is staged in a 4-slot shared-memory ring, so the z
// neighbours come from the ring as well and every field value is loaded (and,
// for the direction kernel, formed) once per tile.  Boundary conditions enter
// only through the halo ("ghost") values: periodic wraps, Dirichlet reads 0,
// Neumann mirrors the boundary value -- which reproduces the corner entries
// (alpha, beta, gamma) of eq. (lap1d) exactly.
#include <cstdio>

#include "tpcg_dev.cuh"

namespace tpcg {

constexpr int TX = 32, TY = 8;
constexpr int SX = TX + 2, SY = TY + 2;

// Map a possibly out-of-range coordinate to the index whose value the ghost
// takes, or -1 for a Dirichlet (zero) ghost.
__device__ __forceinline__ int ghost_index(int g, int n, int bc) {
  if (g >= 0 && g < n) return g;
  if (g == -1) {
    if (bc == kBcP) return n - 1;
    if (bc == kBcN || bc == kBcND) return 0;  // Neumann at the start: mirror
    return -1;                                // Dirichlet at the start
  }
  if (g == n) {
    if (bc == kBcP) return 0;
    if (bc == kBcN || bc == kBcDN) return n - 1;  // Neumann at the end
    return -1;
  }
  return -1;
}

// ------------------------------------------------------------------ fields
struct FieldPlain {  // the stencil is applied to x itself
  const double* __restrict__ x;
  __device__ __forceinline__ double operator()(long long i) const { return __ldg(x + i); }
};

struct FieldDirection {  // FP64 form: P = (Z - mean Z) + beta * P_old   (Algorithm 1; Remark orthogonality)
  const double* __restrict__ z;
  const double* __restrict__ pold;
  double mZ, beta;
  int first;
  __device__ __forceinline__ double operator()(long long i) const {
    const double zi = __ldg(z + i) - mZ;
    return first ? zi : fma(beta, __ldg(pold + i), zi);
  }
};

// ------------------------------------------------------------------ stencil driver
// Calls op(idx, c, w, acc) for every grid point, where c is the field value
// and w = (L field)(point).  Accumulates NQ sums and finishes with fin().
template <int NQ, class Field, class Op, class Fin>
__device__ __forceinline__ void stencil_sweep(const Geom& g, int zchunk, const Field& field, Op& op, double* partials,
                                              unsigned* ticket, Fin fin) {
  __shared__ double ring[4][SY][SX];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * TX + tx;
  const int bx0 = blockIdx.x * TX, by0 = blockIdx.y * TY;
  const int x = bx0 + tx, y = by0 + ty;
  const int k0 = blockIdx.z * zchunk;
  const int k1 = min(g.nz, k0 + zchunk);
  const bool active = (x < g.nx) && (y < g.ny);
  const bool has_z = g.nz > 1;
  const long long plane = (long long)g.nx * g.ny;
  double acc[NQ > 0 ? NQ : 1];
#pragma unroll
  for (int q = 0; q < (NQ > 0 ? NQ : 1); ++q) acc[q] = 0.0;

  auto load_plane = [&](int kk) {
    const int kz = has_z ? ghost_index(kk, g.nz, g.bc[2]) : kk;
    double(*dst)[SX] = ring[kk & 3];
    for (int e = tid; e < SX * SY; e += TX * TY) {
      const int sx = e % SX, sy = e / SX;
      const int gx = ghost_index(bx0 + sx - 1, g.nx, g.bc[0]);
      const int gy = ghost_index(by0 + sy - 1, g.ny, g.bc[1]);
      double v = 0.0;
      if (kz >= 0 && gx >= 0 && gy >= 0 && bx0 + sx - 1 <= g.nx && by0 + sy - 1 <= g.ny)
        v = field((long long)kz * plane + (long long)gy * g.nx + gx);
      dst[sy][sx] = v;
    }
  };

  if (k0 < k1) {
    if (has_z) load_plane(k0 - 1);
    load_plane(k0);
    const double ihx = g.ih2[0], ihy = g.ih2[1], ihz = g.ih2[2];
    const bool uniform = (ihx == ihy) && (!has_z || ihz == ihx);
    for (int k = k0; k < k1; ++k) {
      if (has_z) load_plane(k + 1);
      __syncthreads();
      if (active) {
        const double(*cur)[SX] = ring[k & 3];
        const double c = cur[ty + 1][tx + 1];
        double w;
        if (uniform) {
          double s = (cur[ty + 1][tx] + cur[ty + 1][tx + 2]) + (cur[ty][tx + 1] + cur[ty + 2][tx + 1]);
          double diag = 4.0;
          if (has_z) {
            s += ring[(k - 1) & 3][ty + 1][tx + 1] + ring[(k + 1) & 3][ty + 1][tx + 1];
            diag = 6.0;
          }
          w = fma(diag, c, -s);
          if (ihx != 1.0) w *= ihx;
        } else {
          const double wx = fma(2.0, c, -(cur[ty + 1][tx] + cur[ty + 1][tx + 2]));
          const double wy = fma(2.0, c, -(cur[ty][tx + 1] + cur[ty + 2][tx + 1]));
          w = fma(wx, ihx, wy * ihy);
          if (has_z) {
            const double wz = fma(2.0, c, -(ring[(k - 1) & 3][ty + 1][tx + 1] + ring[(k + 1) & 3][ty + 1][tx + 1]));
            w = fma(wz, ihz, w);
          }
        }
        const long long idx = (long long)k * plane + (long long)y * g.nx + x;
        op(idx, c, w, acc);
      }
    }
  }
  if constexpr (NQ > 0) {
    const int nblocks = gridDim.x * gridDim.y * gridDim.z;
    const int bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    grid_reduce<NQ>(acc, partials, ticket, nblocks, bid, fin);
  }
}

struct NoFin {
  template <class T>
  __device__ void operator()(T&) const {}
};

// ------------------------------------------------------------------ W = L x
struct OpApply {
  double* __restrict__ w;
  __device__ __forceinline__ void operator()(long long i, double, double wv, double (&)[1]) { w[i] = wv; }
};

__global__ void __launch_bounds__(TX* TY) k_apply_laplacian(Geom g, int zchunk, const double* __restrict__ x,
                                                            double* __restrict__ w) {
  FieldPlain f{x};
  OpApply op{w};
  stencil_sweep<0>(g, zchunk, f, op, nullptr, nullptr, NoFin{});
}

// ------------------------------------------------------------------ low-precision copy of R
// Input of the first tensor-core pass: BF16, FP16 of R * 2^shift, TF32, or the
// BF16 pair of R * 2^shift (hi = bf16(R * 2^shift), lo = bf16 of the rest) in two
// planes; rows padded to `pitch` elements.  ptr == nullptr in the FP64 form.
struct LowPrec {
  void* ptr;
  int kind;  // 1 BF16, 2 FP16, 3 TF32 (FP32 containers, rounded to nearest even), 4 BF16 hi/lo planes
  int pitch, nx;
  long long plane;  // kind 4: 16-bit words from the hi plane to the lo plane
};

// The split pair of a value from its FP32 round-to-odd image r32o (= r * 2^shift rounded to odd at 24
// bits): hi = bf16(r32o), which is the correctly rounded bf16(r * 2^shift), and lo = bf16(r32o - hi), the
// difference exact in FP32.  lo equals bf16(r * 2^shift - hi) whenever lo's leading bit lies within 13 bits
// of hi's; below that it may differ from it by one unit of its last place (2^-24 of r), far under the
// pair's 2^-16.  FP32 and conversion arithmetic only: no FP64-pipe work per point.
__device__ __forceinline__ uint32_t f32o_to_bf16_split(float r32o) {
  const __nv_bfloat16 hi = __float2bfloat16_rn(r32o);
  const __nv_bfloat16 lo = __float2bfloat16_rn(r32o - __bfloat162float(hi));
  return (uint32_t)__bfloat16_as_ushort(hi) | ((uint32_t)__bfloat16_as_ushort(lo) << 16);
}

// r -> TF32 in an FP32 container: FP64 -> FP32 round-to-odd on the bit pattern, then round to nearest even
// at the TF32 mantissa (round-to-odd keeps the sticky bit, so the two steps equal one correct rounding).
__device__ __forceinline__ float f64_to_tf32(double r) {
  const uint32_t b = __float_as_uint(f64_to_f32_odd(r, 0));
  if ((b & 0x7f800000u) == 0x7f800000u) return __uint_as_float(b);
  return __uint_as_float((b + 0xfffu + ((b >> 13) & 1u)) & 0xffffe000u);
}

// r32o = f64_to_f32_odd(r, shift): its RNE rounding to FP16 is the correctly
// rounded r * 2^shift, saturated at the FP16 maximum.  BF16 takes r unscaled.
__device__ __forceinline__ void store_lp(const LowPrec& lp, long long i, double r, float r32o) {
  if (!lp.ptr) return;
  long long j = i;
  if (lp.pitch != lp.nx) {  // padded rows (mixed forms: N < 2^32, 32-bit division)
    const unsigned row = (unsigned)i / (unsigned)lp.nx;
    j = (long long)row * lp.pitch + ((unsigned)i - row * (unsigned)lp.nx);
  }
  if (lp.kind == 3) {
    reinterpret_cast<float*>(lp.ptr)[j] = f64_to_tf32(r);
    return;
  }
  if (lp.kind == 4) {
    const uint32_t hl = f32o_to_bf16_split(r32o);
    reinterpret_cast<uint16_t*>(lp.ptr)[j] = (uint16_t)hl;
    reinterpret_cast<uint16_t*>(lp.ptr)[lp.plane + j] = (uint16_t)(hl >> 16);
    return;
  }
  reinterpret_cast<uint16_t*>(lp.ptr)[j] =
      (lp.kind == 2) ? f32_to_f16_bits_rn(fminf(fmaxf(r32o, -65504.0f), 65504.0f)) : f64_to_bf16_bits(r);
}

// Two adjacent values (i even, row pitch even): one packed 4-byte store.
__device__ __forceinline__ void store_lp_pair(const LowPrec& lp, long long i, double r0, double r1, float a32,
                                              float b32) {
  if (!lp.ptr) return;
  long long j = i;
  if (lp.pitch != lp.nx) {  // padded rows (mixed forms: N < 2^32, 32-bit division)
    const unsigned row = (unsigned)i / (unsigned)lp.nx;
    j = (long long)row * lp.pitch + ((unsigned)i - row * (unsigned)lp.nx);
  }
  if (lp.kind == 3) {
    *reinterpret_cast<float2*>(reinterpret_cast<float*>(lp.ptr) + j) = make_float2(f64_to_tf32(r0), f64_to_tf32(r1));
    return;
  }
  if (lp.kind == 4) {
    const uint32_t h0 = f32o_to_bf16_split(a32), h1 = f32o_to_bf16_split(b32);
    uint16_t* q = reinterpret_cast<uint16_t*>(lp.ptr);
    *reinterpret_cast<uint32_t*>(q + j) = (h0 & 0xffffu) | (h1 << 16);
    *reinterpret_cast<uint32_t*>(q + lp.plane + j) = (h0 >> 16) | (h1 & 0xffff0000u);
    return;
  }
  uint32_t v;
  if (lp.kind == 2) {
    const __half2 h = __floats2half2_rn(fminf(fmaxf(a32, -65504.0f), 65504.0f), fminf(fmaxf(b32, -65504.0f), 65504.0f));
    v = *reinterpret_cast<const uint32_t*>(&h);
  } else {
    v = (uint32_t)f64_to_bf16_bits(r0) | ((uint32_t)f64_to_bf16_bits(r1) << 16);
  }
  *reinterpret_cast<uint32_t*>(reinterpret_cast<uint16_t*>(lp.ptr) + j) = v;
}

// ------------------------------------------------------------------ fixed-point stencil driver
// Same 32 x 8 tiles and 4-slot plane ring as stencil_sweep, for fields held as
// exact integers (IT = int or long long), organised for memory-level
// parallelism:
//  * persistent and balanced: the (tile, plane) pairs are numbered tile-major
//    and block b takes a contiguous range of T / G or T / G + 1 of them,
//    walked as one or two runs of consecutive planes of a tile;
//  * software-pipelined, two planes per block barrier: the global loads of
//    ring planes k+3 and k+4 (Field::load, raw values in registers) and of the
//    per-point operands of planes k+2 and k+3 (Op::load) are issued before the
//    barrier of planes k and k+1, so their latency overlaps the work on those
//    two planes; Field::convert forms the integer value when the raw values
//    are committed to the ring.  With six slots the commits of planes k+3 and
//    k+4 never touch a slot that a thread still on planes k and k+1 reads.
// op(i, x, y, k, pre, c, xl, xr, yl, yr, zl, zr) receives the point value and
// its six neighbours with the ghosts applied (zl = zr = c in 2D), so every
// second difference is exact.  op.flush(acc) turns the op's own per-thread
// sums into the NQ doubles of the deterministic grid reduction.
template <class IT, int NQ, class Field, class Op, class Fin>
__device__ __forceinline__ void stencil_sweep_fx(const Geom& g, const Field& field, Op& op, double* partials,
                                                 unsigned* ticket, Fin fin) {
  constexpr int NT = TX * TY;
  constexpr int PER = (SX * SY + NT - 1) / NT;
  __shared__ IT ring[6][SY][SX];
  using Raw = typename Field::Raw;
  using Pre = typename Op::Pre;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * TX + tx;
  const bool has_z = g.nz > 1;
  // N <= 2^31: every index and count fits in 32 bits.  All index arithmetic
  // stays in 32-bit integers (64-bit division is emulated on the FP64 pipe).
  const unsigned plane = (unsigned)g.nx * (unsigned)g.ny;
  const unsigned bxn = (unsigned)(g.nx + TX - 1) / TX, byn = (unsigned)(g.ny + TY - 1) / TY;
  const unsigned T = bxn * byn * (unsigned)g.nz;
  const unsigned G = gridDim.x, q = T / G, rm = T - q * G;  // block b: q + (b < rm) consecutive pairs
  const unsigned t_begin = blockIdx.x * q + min(blockIdx.x, rm);
  const unsigned t_end = t_begin + q + (blockIdx.x < rm ? 1u : 0u);
  Raw rawA[PER], rawB[PER];
  unsigned off[PER];
  bool okxy[PER];
  for (unsigned t = t_begin; t < t_end;) {
    const unsigned tile = t / (unsigned)g.nz;
    const int k0 = (int)(t - tile * (unsigned)g.nz);
    const int k1 = (int)min((unsigned)g.nz, (unsigned)k0 + (t_end - t));
    t += (unsigned)(k1 - k0);
    const unsigned tyi = tile / bxn;
    const int bx0 = (int)(tile - tyi * bxn) * TX, by0 = (int)tyi * TY;
    const int x = bx0 + tx, y = by0 + ty;
    const bool active = (x < g.nx) && (y < g.ny);
#pragma unroll
    for (int j = 0; j < PER; ++j) {
      const int e = tid + j * NT;
      const int gx = ghost_index(bx0 + e % SX - 1, g.nx, g.bc[0]);
      const int gy = ghost_index(by0 + e / SX - 1, g.ny, g.bc[1]);
      okxy[j] = (e < SX * SY) && gx >= 0 && gy >= 0;
      off[j] = (unsigned)gy * (unsigned)g.nx + (unsigned)gx;
    }
    auto slot = [](int kk) { return (kk + 6) % 6; };  // kk >= -1
    auto issue = [&](Raw(&raw)[PER], int kk) {
      const int kz = has_z ? ghost_index(kk, g.nz, g.bc[2]) : kk;
#pragma unroll
      for (int j = 0; j < PER; ++j) raw[j] = (okxy[j] && kz >= 0) ? field.load((unsigned)kz * plane + off[j]) : Raw{};
    };
    auto commit = [&](const Raw(&raw)[PER], int kk) {
      IT(*dst)[SX] = ring[slot(kk)];
#pragma unroll
      for (int j = 0; j < PER; ++j) {
        const int e = tid + j * NT;
        if (e < SX * SY) dst[e / SX][e % SX] = field.convert(raw[j]);
      }
    };
    const unsigned col = (unsigned)y * (unsigned)g.nx + (unsigned)x;
    __syncthreads();  // the previous run's last planes have been consumed
    if (has_z) {
      issue(rawA, k0 - 1);
      commit(rawA, k0 - 1);
    }
    issue(rawA, k0);
    commit(rawA, k0);
    if (has_z) {
      issue(rawA, k0 + 1);
      if (k0 + 1 < k1) issue(rawB, k0 + 2);
    }
    Pre pre0 = active ? op.load((unsigned)k0 * plane + col) : Pre{};
    Pre pre1 = (active && k0 + 1 < k1) ? op.load((unsigned)(k0 + 1) * plane + col) : Pre{};
    auto point = [&](int k, const Pre& pre) {
      const IT(*cur)[SX] = ring[slot(k)];
      const IT c = cur[ty + 1][tx + 1];
      const IT zl = has_z ? ring[slot(k - 1)][ty + 1][tx + 1] : c;
      const IT zr = has_z ? ring[slot(k + 1)][ty + 1][tx + 1] : c;
      op((unsigned)k * plane + col, x, y, k, pre, c, cur[ty + 1][tx], cur[ty + 1][tx + 2], cur[ty][tx + 1],
         cur[ty + 2][tx + 1], zl, zr);
    };
    // two planes per block barrier: planes k and k+1 read ring planes k-1 .. k+2; the commits of k+3 and k+4
    // (next step, before its barrier) go to the two other slots of the six
    for (int k = k0; k < k1; k += 2) {
      const bool two = k + 1 < k1;
      if (has_z) {
        commit(rawA, k + 1);
        if (two) commit(rawB, k + 2);
        if (k + 2 < k1) issue(rawA, k + 3);
        if (k + 3 < k1) issue(rawB, k + 4);
      }
      Pre next0{}, next1{};
      if (active && k + 2 < k1) next0 = op.load((unsigned)(k + 2) * plane + col);
      if (active && k + 3 < k1) next1 = op.load((unsigned)(k + 3) * plane + col);
      __syncthreads();
      if (active) {
        point(k, pre0);
        if (two) point(k + 1, pre1);
      }
      pre0 = next0;
      pre1 = next1;
    }
  }
  double acc[NQ];
  op.flush(acc);
  grid_reduce<NQ>(acc, partials, ticket, gridDim.x, blockIdx.x, fin);
}

struct NoPre {};

// max |U| is tracked on FP64 bit patterns shifted left by one: dropping the
// sign bit this way keeps the order of magnitudes and stays an integer
// operation (a sign-bit mask would be turned into an FP64 absolute value,
// which issues on the slow FP64 pipe).  Thread 0 folds the block's maximum
// into the state's accumulator; order-independent, so deterministic.
__device__ __forceinline__ unsigned long long mag_key(double u) {
  return (unsigned long long)__double_as_longlong(u) << 1;
}
__device__ __forceinline__ void fold_umax(SolveState* st, unsigned long long um) {
  const unsigned long long m = block_max_u64(um);
  if (threadIdx.x + threadIdx.y == 0) atomicMax(&st->umax_bits, m >> 1);
}

// ------------------------------------------------------------------ residual R = eta_hat - L U
// The initial residual (Algorithm 1) and the check of the true
// residual behind the stop test (Remark stoppincrit).  U enters as exact
// int64 fixed point round(U * 2^ku), max|U| * 2^ku < 2^58, so the stencil
// is exact and W = L U is rounded to FP64 once; r = eta_hat - W is one more
// rounding (an FMA with the 1/h^2 weight).  The quantisation of U is below
// 2^-58 max|U|, under the FP64 rounding of U's largest entries.  The check
// replaces R by the true residual (residual replacement) and sums U for the
// exit centring; ||r||^2 and sum(r) are accumulated per thread in FP32 from
// r * 2^sr, where 2^-sr bounds every |r|.
template <bool INIT>
struct OpResidualFx {
  using Pre = double;  // eta at the point
  __device__ __forceinline__ double load(unsigned i) const { return __ldg(eta + i); }
  const double* __restrict__ eta;
  double* __restrict__ R;
  LowPrec lp;
  double mean, nih0, nih1, nih2;  // -1/h^2 per axis
  int shift, sr, ku, uniform;
  float rr, sR;
  double ee;  // ||eta_hat||^2 in FP64: it scales the tolerance and is reported
  long long su;
  __device__ __forceinline__ void operator()(unsigned i, int, int, int, double eta_i, long long c, long long xl,
                                             long long xr, long long yl, long long yr, long long zl, long long zr) {
    const long long dx = 2 * c - xl - xr, dy = 2 * c - yl - yr, dz = 2 * c - zl - zr;
    const double e = eta_i - mean;
    double r;
    if (uniform) {
      r = fma(nih0, i64_to_f64_scaled_hw(dx + dy + dz, -ku), e);
    } else {
      r = fma(nih0, i64_to_f64_scaled(dx, -ku), e);
      r = fma(nih1, i64_to_f64_scaled(dy, -ku), r);
      if (dz) r = fma(nih2, i64_to_f64_scaled(dz, -ku), r);
    }
    R[i] = r;
    store_lp(lp, i, r, f64_to_f32_odd(r, shift));
    const float r32 = f64_to_f32_odd(r, sr);
    rr = fmaf(r32, r32, rr);
    sR += r32;
    if (INIT) ee = fma(e, e, ee);
    su += c >> 8;  // |c| < 2^58: a thread's sum of fewer than 2^13 terms stays inside int64
  }
  __device__ __forceinline__ void flush(double (&acc)[4]) {
    acc[0] = f32_to_f64_int(rr);
    acc[1] = f32_to_f64_int(sR);
    acc[2] = i64_to_f64_scaled(su, 0);
    acc[3] = ee;
  }
};

struct FieldFixed64 {  // U -> round(U * 2^k)
  using Raw = double;
  const double* __restrict__ u;
  int k;
  __device__ __forceinline__ double load(unsigned i) const { return __ldg(u + i); }
  __device__ __forceinline__ long long convert(double v) const { return f64_to_fixed64(v, k); }
};

// The low-precision copy just written used lp_shift; the next one uses the
// exponent that scales the new residual to unit RMS.
__device__ __forceinline__ void advance_shift(SolveState* st, double rr, long long N) {
  st->lp_shift_applied = st->lp_shift;
  st->lp_shift = lp_shift_for(rr, N);
}

// s = {||R_0||^2, sum(R_0), ||eta_hat||^2}
__device__ void fin_init(SolveState* st, const double (&s)[3], long long N) {
  st->rr = s[0];
  st->sumR = s[1];
  st->eta_norm2 = s[2];
  st->tol2 = st->tol2 * s[2];  // tol^2 was stored; scale by ||eta_hat||^2
  advance_shift(st, s[0], N);
  if (!isfinite(s[0]) || !isfinite(s[2])) {
    st->status = TPCG_ERR_BREAKDOWN;
    st->done = 1;
  } else if (s[2] == 0.0) {  // eta_hat = 0: the minimum-norm solution is 0
    st->status = TPCG_OK;
    st->done = 2;
  }
}

// s = {||eta_hat - L U||^2, sum(eta_hat - L U), sum(U)}
__device__ void fin_true(SolveState* st, const double (&s)[3], long long N) {
  st->true_rr = s[0];
  st->sumU = s[2];
  advance_shift(st, s[0], N);
  if (!isfinite(s[0])) {
    st->status = TPCG_ERR_BREAKDOWN;
    st->done = 1;
    return;
  }
  if (s[0] <= st->tol2) {
    st->status = TPCG_OK;
    st->done = 1;
    st->done_iter = st->iter;
  } else if (st->iter >= st->maxit) {
    st->status = TPCG_ERR_NOT_CONVERGED;
    st->done = 1;
  } else {  // keep iterating from the replaced (true) residual
    st->rr = s[0];
    st->sumR = s[1];
    st->need_check = 0;
  }
}

// INIT: R_0 = eta_hat - L U_0 for a given U_0 (max|U_0| from k_eta_sum).
// Otherwise the stop-test check; `force` evaluates the residual of the
// returned iterate for the report only.
template <bool INIT>
__global__ void __launch_bounds__(TX* TY) k_residual_fx(Geom g, const double* __restrict__ eta,
                                                        const double* __restrict__ U, double* __restrict__ R,
                                                        LowPrec lp, SolveState* st, double* partials, int force) {
  if (!INIT && !force && (st->done || !st->need_check)) return;
  // the solve's buffers come from the state (a captured launch sequence serves every solve of the plan)
  eta = st->eta;
  U = st->ups;
  const int ku = st->ku, sr = st->sr;
  FieldFixed64 f{U, ku};
  OpResidualFx<INIT> op{eta, R, lp, st->mean_eta, g.nih2[0], g.nih2[1], g.nih2[2], st->lp_shift, sr, ku, g.uniform,
                        0.0f, 0.0f, 0.0, 0};
  const long long N = g.N;
  const bool finite_u = isfinite(st->umax);
  stencil_sweep_fx<long long, 4>(
      g, f, op, partials, &st->tickets[INIT ? kTkInit : kTkTrue],
      [st, force, N, sr, ku, finite_u](const double(&s)[4]) {
        const double rr = finite_u ? ldexp(s[0], -2 * sr) : __longlong_as_double(0x7ff8000000000000ll);
        const double sumR = ldexp(s[1], -sr), sumU = ldexp(s[2], 8 - ku);
        if (!INIT) st->checks += 1;
        if (INIT) {
          const double v[3] = {rr, sumR, s[3]};
          fin_init(st, v, N);
        } else if (force) {
          st->true_rr = rr;
          st->sumU = sumU;
        } else {
          const double v[3] = {rr, sumR, sumU};
          fin_true(st, v, N);
        }
      });
}

// ------------------------------------------------------------------ direction + W = L P (FP64 form)
// P_s = Z_s' + beta_s P_{s-1} (Algorithm 1, with Z centred), W = L P, <W, P>
// and the step length alpha = rho / <W, P>.
struct OpDirection {
  double* __restrict__ P;
  double* __restrict__ W;
  __device__ __forceinline__ void operator()(long long i, double c, double w, double (&acc)[1]) {
    P[i] = c;
    W[i] = w;
    acc[0] = fma(w, c, acc[0]);
  }
};

__device__ void fin_direction(SolveState* st, const double (&s)[1], const Geom& g) {
  st->pWp = s[0];
  st->first = 0;
  if (!(s[0] > 0.0) || !isfinite(s[0])) {
    st->status = TPCG_ERR_BREAKDOWN;
    st->done = 1;
    return;
  }
  const double alpha = st->rho / s[0];
  st->alpha = alpha;
  for (int m = 0; m < 3; ++m) st->nah[m] = -alpha * g.ih2[m];
}

__global__ void __launch_bounds__(TX* TY) k_direction(Geom g, int zchunk, const double* __restrict__ Z,
                                                      const double* __restrict__ Pold, double* __restrict__ P,
                                                      double* __restrict__ W, SolveState* st, double* partials) {
  if (st->done) return;
  FieldDirection f{Z, Pold, st->mZ, st->beta, st->first};
  OpDirection op{P, W};
  stencil_sweep<1>(g, zchunk, f, op, partials, &st->tickets[kTkDir],
                   [st, g](const double(&s)[1]) { fin_direction(st, s, g); });
}

// ------------------------------------------------------------------ direction, mixed forms
// Z arrives in FP32.  The direction is stored as exact fixed point
//     P_s = 2^-kp P_int,   P_int = round((Z_s + beta_s P_{s-1}) 2^kp),  |P_int| <= 2^20,
// (Algorithm 1), with kp from the bound max|Z_s| + |beta_s| max|P_{s-1}|.
// W_s = L P_s is never stored: it is an exact integer stencil of
// P_int, recomputed where it is needed, so U += alpha P and R -= alpha W stay
// consistent with one another whatever the rounding of P_s was.  The
// step-length denominator <W_s, P_s> = <L P_s, P_s> is summed in its edge form: by
// summation by parts on eq. (lap1d), <L_n p, p> is the sum of (p_i - p_{i-1})^2
// over the edges of the axis, the start edge taken to the ghost value
// (periodic: the wrapped neighbour; Dirichlet: 0; Neumann: itself) plus, for a
// Dirichlet end, the end edge p_{n-1}^2.  Every term is non-negative, so the
// FP32 sum of exact integer squares has no cancellation.  P_s
// keeps the constant (null-space) component of Z: L annihilates it, so W and
// <W, P> are those of the centred Z (Remark orthogonality), rho is corrected
// by -mean(Z) sum(R), and the constant offset of U is removed at exit.
// Register-window streams.  Thread (tx, ty) of a 32 x 8 block owns the grid
// column (x, y) of a tile and marches in z: its z neighbours stay in
// registers, x neighbours come from the neighbouring lanes by warp shuffle
// (lanes 0 and 31 fetch the tile's halo column themselves), y neighbours from
// loads of the rows the other warps stream (cache hits).  No shared memory and
// no block barrier per plane.  Blocks take balanced contiguous ranges of
// (tile, plane) pairs, walked as runs of consecutive planes of one tile.
// Ghosts: ghost_index() maps a neighbour across a boundary to the wrapped
// index (P), the point itself (N: mirror) or -1 (D: the value 0).
template <int TW = TX, class Run>
__device__ __forceinline__ void for_each_run(const Geom& g, Run run) {
  const unsigned bxn = (unsigned)(g.nx + TW - 1) / TW, byn = (unsigned)(g.ny + TY - 1) / TY;
  const unsigned T = bxn * byn * (unsigned)g.nz;
  const unsigned G = gridDim.x, q = T / G, rm = T - q * G;
  const unsigned t_begin = blockIdx.x * q + min(blockIdx.x, rm);
  const unsigned t_end = t_begin + q + (blockIdx.x < rm ? 1u : 0u);
  for (unsigned t = t_begin; t < t_end;) {
    const unsigned tile = t / (unsigned)g.nz;
    const int k0 = (int)(t - tile * (unsigned)g.nz);
    const int k1 = (int)min((unsigned)g.nz, (unsigned)k0 + (t_end - t));
    t += (unsigned)(k1 - k0);
    const unsigned tyi = tile / bxn;
    run((int)(tile - tyi * bxn) * TW, (int)tyi * TY, k0, k1);
  }
}

__global__ void __launch_bounds__(TX* TY) k_direction_int(Geom g, const float* __restrict__ Z,
                                                          const int* __restrict__ Pold, int* __restrict__ P,
                                                          SolveState* st, double* partials) {
  if (st->done) return;
  const int kp = st->kp_next;
  const float sc = (kp >= -126 && kp <= 127) ? __int_as_float((kp + 127) << 23) : 0.0f;  // 2^kp
  const float bs = st->bs_next;  // beta_s 2^-kp_{s-1} (0 for the first direction)
  const int first = st->first;
  const unsigned nx = (unsigned)g.nx, plane = (unsigned)g.nx * (unsigned)g.ny;
  const bool has_z = g.nz > 1;
  // P_int formed from Z_s and P_{s-1} at one grid point
  struct Raw {
    float z;
    int p;
  };
  auto load = [&](unsigned i) -> Raw { return Raw{__ldg(Z + i), first ? 0 : __ldg(Pold + i)}; };
  auto form = [&](Raw r) -> int {
    const float v = fmaf(bs, i22_to_f32(r.p), r.z);
    return sc != 0.0f ? f32_to_i22(v, sc) : f32_to_fixed(v, kp);  // 2^kp outside the FP32 range: integer path
  };
  // the end edge of an axis counts only for a Dirichlet end (ghost 0; a Neumann ghost gives a zero edge)
  const bool endx = g.bc[0] == kBcD || g.bc[0] == kBcND, endy = g.bc[1] == kBcD || g.bc[1] == kBcND;
  const bool endz = has_z && (g.bc[2] == kBcD || g.bc[2] == kBcND);
  const float w0 = g.ih2f[0], w1 = g.ih2f[1], w2 = g.ih2f[2];
  const int lane = threadIdx.x;
  float e = 0.0f;
  int pm = 0;
  constexpr int UZ = 4;  // planes whose loads are issued together (memory-level parallelism)
  for_each_run(g, [&](int bx0, int by0, int k0, int k1) {
    const int x = bx0 + lane, y = by0 + threadIdx.y;
    const bool active = x < g.nx && y < g.ny;
    const int xg = ghost_index(x - 1, g.nx, g.bc[0]);  // used by lane 0 (the tile's left halo)
    const int yg = ghost_index(y - 1, g.ny, g.bc[1]);
    const bool has_xl = lane == 0 && active && xg >= 0, has_yl = active && yg >= 0;
    // in-plane offsets; inactive or absent neighbours read a valid point and discard the value
    const unsigned col = active ? (unsigned)y * nx + (unsigned)x : 0u;
    const unsigned colx = has_xl ? (unsigned)y * nx + (unsigned)xg : col;
    const unsigned coly = has_yl ? (unsigned)yg * nx + (unsigned)x : col;
    int zprev = 0;
    if (has_z && active) {
      const int kz = ghost_index(k0 - 1, g.nz, g.bc[2]);
      zprev = kz >= 0 ? form(load((unsigned)kz * plane + col)) : 0;
    }
    for (int kb = k0; kb < k1; kb += UZ) {
      Raw own[UZ], up[UZ], left[UZ];
#pragma unroll
      for (int j = 0; j < UZ; ++j) {
        const unsigned base = (unsigned)min(kb + j, k1 - 1) * plane;
        own[j] = load(base + col);
        up[j] = load(base + coly);
        left[j] = load(base + colx);
      }
#pragma unroll
      for (int j = 0; j < UZ; ++j) {
        const int k = kb + j;
        if (k >= k1) break;  // block-uniform
        const int c = active ? form(own[j]) : 0;
        int xl = __shfl_up_sync(0xffffffffu, c, 1);
        if (lane == 0) xl = has_xl ? form(left[j]) : 0;
        const int yl = has_yl ? form(up[j]) : 0;
        const int zl = has_z ? zprev : c;
        if (active) {
          P[(unsigned)k * plane + col] = c;
          pm = max(pm, abs(c));
          const float dx = i22_to_f32(c - xl), dy = i22_to_f32(c - yl), dz = i22_to_f32(c - zl);
          float tx = dx * dx, ty = dy * dy, tz = dz * dz;
          const float cf = i22_to_f32(c);
          if (endx && x == g.nx - 1) tx = fmaf(cf, cf, tx);
          if (endy && y == g.ny - 1) ty = fmaf(cf, cf, ty);
          if (endz && k == g.nz - 1) tz = fmaf(cf, cf, tz);
          e = fmaf(w0, tx, fmaf(w1, ty, fmaf(w2, tz, e)));
        }
        zprev = c;
      }
    }
  });
  double acc[1] = {f32_to_f64_int(e)};
  const unsigned long long m = block_max_u64((unsigned long long)pm);
  if (threadIdx.x + threadIdx.y == 0) atomicMax(&st->pmax_bits, (unsigned)m);
  const int nblocks = gridDim.x;
  grid_reduce<1>(acc, partials, &st->tickets[kTkDir], nblocks, blockIdx.x, [st, kp, g](const double(&s)[1]) {
    st->kp = kp;
    st->pmax = ldexp((double)atomicExch(&st->pmax_bits, 0u), -kp);
    const double v[1] = {ldexp(s[0], -2 * kp)};
    fin_direction(st, v, g);
  });
}

// The same direction with two adjacent x points per thread (even nx): Z and
// P_old as 8-byte pairs, P stored as int2; the left neighbour of a pair's
// first point comes from the previous lane (lane 0: the tile's halo column).
__global__ void __launch_bounds__(TX* TY) k_direction_pair(Geom g, const float* __restrict__ Z,
                                                           const int* __restrict__ Pold, int* __restrict__ P,
                                                           SolveState* st, double* partials) {
  if (st->done) return;
  const int kp = st->kp_next;
  const float sc = (kp >= -126 && kp <= 127) ? __int_as_float((kp + 127) << 23) : 0.0f;  // 2^kp
  const float bs = st->bs_next;  // beta_s 2^-kp_{s-1} (0 for the first direction)
  const int first = st->first;
  const unsigned nx = (unsigned)g.nx, plane = (unsigned)g.nx * (unsigned)g.ny;
  const bool has_z = g.nz > 1;
  struct Raw2 {
    float2 z;
    int2 p;
  };
  auto load2 = [&](unsigned i) -> Raw2 {
    return Raw2{__ldg(reinterpret_cast<const float2*>(Z + i)),
                first ? make_int2(0, 0) : __ldg(reinterpret_cast<const int2*>(Pold + i))};
  };
  auto form1 = [&](float z, int po) -> int {
    const float v = fmaf(bs, i22_to_f32(po), z);
    return sc != 0.0f ? f32_to_i22(v, sc) : f32_to_fixed(v, kp);  // 2^kp outside the FP32 range: integer path
  };
  const bool endx = g.bc[0] == kBcD || g.bc[0] == kBcND, endy = g.bc[1] == kBcD || g.bc[1] == kBcND;
  const bool endz = has_z && (g.bc[2] == kBcD || g.bc[2] == kBcND);
  const float w0 = g.ih2f[0], w1 = g.ih2f[1], w2 = g.ih2f[2];
  const int lane = threadIdx.x;
  float e = 0.0f;
  int pm = 0;
  constexpr int UZ = 2;  // planes whose loads are issued together
  for_each_run<2 * TX>(g, [&](int bx0, int by0, int k0, int k1) {
    const int x = bx0 + 2 * lane, y = by0 + threadIdx.y;
    const bool active = x < g.nx && y < g.ny;  // nx even: both points or neither
    const int xg = ghost_index(x - 1, g.nx, g.bc[0]);
    const int yg = ghost_index(y - 1, g.ny, g.bc[1]);
    const bool has_xl = lane == 0 && active && xg >= 0, has_yl = active && yg >= 0;
    const unsigned col = active ? (unsigned)y * nx + (unsigned)x : 0u;
    const unsigned colx = has_xl ? (unsigned)y * nx + (unsigned)xg : col;
    const unsigned coly = has_yl ? (unsigned)yg * nx + (unsigned)x : col;
    const bool last_x = x + 1 == g.nx - 1;
    int2 zprev = make_int2(0, 0);
    if (has_z && active) {
      const int kz = ghost_index(k0 - 1, g.nz, g.bc[2]);
      if (kz >= 0) {
        const Raw2 r = load2((unsigned)kz * plane + col);
        zprev = make_int2(form1(r.z.x, r.p.x), form1(r.z.y, r.p.y));
      }
    }
    for (int kb = k0; kb < k1; kb += UZ) {
      Raw2 own[UZ], up[UZ];
      float lz[UZ];
      int lp[UZ];
#pragma unroll
      for (int j = 0; j < UZ; ++j) {
        const unsigned base = (unsigned)min(kb + j, k1 - 1) * plane;
        own[j] = load2(base + col);
        up[j] = load2(base + coly);
        lz[j] = __ldg(Z + base + colx);
        lp[j] = first ? 0 : __ldg(Pold + base + colx);
      }
#pragma unroll
      for (int j = 0; j < UZ; ++j) {
        const int k = kb + j;
        if (k >= k1) break;  // block-uniform
        int2 c = make_int2(0, 0);
        if (active) c = make_int2(form1(own[j].z.x, own[j].p.x), form1(own[j].z.y, own[j].p.y));
        int xl = __shfl_up_sync(0xffffffffu, c.y, 1);
        if (lane == 0) xl = has_xl ? form1(lz[j], lp[j]) : 0;
        const int2 yl = has_yl ? make_int2(form1(up[j].z.x, up[j].p.x), form1(up[j].z.y, up[j].p.y))
                               : make_int2(0, 0);
        const int2 zl = has_z ? zprev : c;
        if (active) {
          *reinterpret_cast<int2*>(P + (unsigned)k * plane + col) = c;
          pm = max(pm, max(abs(c.x), abs(c.y)));
          const float dx0 = i22_to_f32(c.x - xl), dx1 = i22_to_f32(c.y - c.x);
          const float dy0 = i22_to_f32(c.x - yl.x), dy1 = i22_to_f32(c.y - yl.y);
          const float dz0 = i22_to_f32(c.x - zl.x), dz1 = i22_to_f32(c.y - zl.y);
          float tx = fmaf(dx0, dx0, dx1 * dx1), ty = fmaf(dy0, dy0, dy1 * dy1), tz = fmaf(dz0, dz0, dz1 * dz1);
          const float cf0 = i22_to_f32(c.x), cf1 = i22_to_f32(c.y);
          if (endx && last_x) tx = fmaf(cf1, cf1, tx);
          if (endy && y == g.ny - 1) ty = fmaf(cf0, cf0, fmaf(cf1, cf1, ty));
          if (endz && k == g.nz - 1) tz = fmaf(cf0, cf0, fmaf(cf1, cf1, tz));
          e = fmaf(w0, tx, fmaf(w1, ty, fmaf(w2, tz, e)));
        }
        zprev = c;
      }
    }
  });
  double acc[1] = {f32_to_f64_int(e)};
  const unsigned long long m = block_max_u64((unsigned long long)pm);
  if (threadIdx.x + threadIdx.y == 0) atomicMax(&st->pmax_bits, (unsigned)m);
  grid_reduce<1>(acc, partials, &st->tickets[kTkDir], gridDim.x, blockIdx.x, [st, kp, g](const double(&s)[1]) {
    st->kp = kp;
    st->pmax = ldexp((double)atomicExch(&st->pmax_bits, 0u), -kp);
    const double v[1] = {ldexp(s[0], -2 * kp)};
    fin_direction(st, v, g);
  });
}

// The same direction with four adjacent x points per thread (nx a multiple of
// 4): Z and P_old as 16-byte quads, P stored as int4; the left neighbour of a
// quad's first point comes from the previous lane (lane 0: the tile's halo
// column).  Loads, address arithmetic and loop control are shared by four
// points instead of two.
__global__ void __launch_bounds__(TX* TY) k_direction_quad(Geom g, const float* __restrict__ Z,
                                                           const int* __restrict__ Pold, int* __restrict__ P,
                                                           SolveState* st, double* partials) {
  if (st->done) return;
  const int kp = st->kp_next;
  const float sc = (kp >= -126 && kp <= 127) ? __int_as_float((kp + 127) << 23) : 0.0f;  // 2^kp
  const float bs = st->bs_next;  // beta_s 2^-kp_{s-1} (0 for the first direction)
  const int first = st->first;
  const unsigned nx = (unsigned)g.nx, plane = (unsigned)g.nx * (unsigned)g.ny;
  const bool has_z = g.nz > 1;
  struct Raw4 {
    float4 z;
    int4 p;
  };
  auto load4 = [&](unsigned i) -> Raw4 {
    return Raw4{__ldg(reinterpret_cast<const float4*>(Z + i)),
                first ? make_int4(0, 0, 0, 0) : __ldg(reinterpret_cast<const int4*>(Pold + i))};
  };
  const bool endx = g.bc[0] == kBcD || g.bc[0] == kBcND, endy = g.bc[1] == kBcD || g.bc[1] == kBcND;
  const bool endz = has_z && (g.bc[2] == kBcD || g.bc[2] == kBcND);
  const float w0 = g.ih2f[0], w1 = g.ih2f[1], w2 = g.ih2f[2];
  const int lane = threadIdx.x;
  float e = 0.0f;
  int pm = 0;
  constexpr int UZ = 2;  // planes whose loads are issued together
  // the sweep, instantiated for 2^kp inside the FP32 range (one FMA per rounding) and outside it (integer
  // path), so that the per-point code carries one of them only
  auto sweep = [&](auto fast) {
  constexpr bool kFast = decltype(fast)::value;
  auto form1 = [&](float z, int po) -> int {
    const float v = fmaf(bs, i22_to_f32(po), z);
    if constexpr (kFast) return f32_to_i22(v, sc);
    else return f32_to_fixed(v, kp);
  };
  auto form4 = [&](const Raw4& r) -> int4 {
    return make_int4(form1(r.z.x, r.p.x), form1(r.z.y, r.p.y), form1(r.z.z, r.p.z), form1(r.z.w, r.p.w));
  };
  for_each_run<4 * TX>(g, [&](int bx0, int by0, int k0, int k1) {
    const int x = bx0 + 4 * lane, y = by0 + threadIdx.y;
    const bool active = x < g.nx && y < g.ny;  // nx a multiple of 4: all four points or none
    const int xg = ghost_index(x - 1, g.nx, g.bc[0]);
    const int yg = ghost_index(y - 1, g.ny, g.bc[1]);
    const bool has_xl = lane == 0 && active && xg >= 0, has_yl = active && yg >= 0;
    const unsigned col = active ? (unsigned)y * nx + (unsigned)x : 0u;
    const unsigned colx = has_xl ? (unsigned)y * nx + (unsigned)xg : col;
    const unsigned coly = has_yl ? (unsigned)yg * nx + (unsigned)x : col;
    const bool last_x = x + 3 == g.nx - 1;
    int4 zprev = make_int4(0, 0, 0, 0);
    if (has_z && active) {
      const int kz = ghost_index(k0 - 1, g.nz, g.bc[2]);
      if (kz >= 0) zprev = form4(load4((unsigned)kz * plane + col));
    }
    for (int kb = k0; kb < k1; kb += UZ) {
      Raw4 own[UZ], up[UZ];
      float lz[UZ];
      int lp[UZ];
#pragma unroll
      for (int j = 0; j < UZ; ++j) {
        const unsigned base = (unsigned)min(kb + j, k1 - 1) * plane;
        own[j] = load4(base + col);
        up[j] = load4(base + coly);
        lz[j] = __ldg(Z + base + colx);
        lp[j] = first ? 0 : __ldg(Pold + base + colx);
      }
#pragma unroll
      for (int j = 0; j < UZ; ++j) {
        const int k = kb + j;
        if (k >= k1) break;  // block-uniform
        int4 c = make_int4(0, 0, 0, 0);
        if (active) c = form4(own[j]);
        int xl = __shfl_up_sync(0xffffffffu, c.w, 1);
        if (lane == 0) xl = has_xl ? form1(lz[j], lp[j]) : 0;
        const int4 yl = has_yl ? form4(up[j]) : make_int4(0, 0, 0, 0);
        const int4 zl = has_z ? zprev : c;
        if (active) {
          *reinterpret_cast<int4*>(P + (unsigned)k * plane + col) = c;
          pm = max(pm, max(max(abs(c.x), abs(c.y)), max(abs(c.z), abs(c.w))));
          const float dx0 = i22_to_f32(c.x - xl), dx1 = i22_to_f32(c.y - c.x), dx2 = i22_to_f32(c.z - c.y),
                      dx3 = i22_to_f32(c.w - c.z);
          const float dy0 = i22_to_f32(c.x - yl.x), dy1 = i22_to_f32(c.y - yl.y), dy2 = i22_to_f32(c.z - yl.z),
                      dy3 = i22_to_f32(c.w - yl.w);
          const float dz0 = i22_to_f32(c.x - zl.x), dz1 = i22_to_f32(c.y - zl.y), dz2 = i22_to_f32(c.z - zl.z),
                      dz3 = i22_to_f32(c.w - zl.w);
          float tx = fmaf(dx0, dx0, fmaf(dx1, dx1, fmaf(dx2, dx2, dx3 * dx3)));
          float ty = fmaf(dy0, dy0, fmaf(dy1, dy1, fmaf(dy2, dy2, dy3 * dy3)));
          float tz = fmaf(dz0, dz0, fmaf(dz1, dz1, fmaf(dz2, dz2, dz3 * dz3)));
          if (endx && last_x) {
            const float cf = i22_to_f32(c.w);
            tx = fmaf(cf, cf, tx);
          }
          if ((endy && y == g.ny - 1) || (endz && k == g.nz - 1)) {
            const float c0 = i22_to_f32(c.x), c1 = i22_to_f32(c.y), c2 = i22_to_f32(c.z), c3 = i22_to_f32(c.w);
            const float sq = fmaf(c0, c0, fmaf(c1, c1, fmaf(c2, c2, c3 * c3)));
            if (endy && y == g.ny - 1) ty += sq;
            if (endz && k == g.nz - 1) tz += sq;
          }
          e = fmaf(w0, tx, fmaf(w1, ty, fmaf(w2, tz, e)));
        }
        zprev = c;
      }
    }
  });
  };
  if (sc != 0.0f) sweep(std::true_type{});
  else sweep(std::false_type{});
  double acc[1] = {f32_to_f64_int(e)};
  const unsigned long long m = block_max_u64((unsigned long long)pm);
  if (threadIdx.x + threadIdx.y == 0) atomicMax(&st->pmax_bits, (unsigned)m);
  grid_reduce<1>(acc, partials, &st->tickets[kTkDir], gridDim.x, blockIdx.x, [st, kp, g](const double(&s)[1]) {
    st->kp = kp;
    st->pmax = ldexp((double)atomicExch(&st->pmax_bits, 0u), -kp);
    const double v[1] = {ldexp(s[0], -2 * kp)};
    fin_direction(st, v, g);
  });
}

// ------------------------------------------------------------------ update
// U += alpha P and R -= alpha W (Algorithm 1), low-precision copy of R,
// ||R||^2 and sum(R) for the stop test and the centring correction of rho,
// and max|U| for the fixed-point residual check.  The two sums are
// accumulated per thread in FP32 from R * 2^lp_shift (exact
// power-of-two scaling, unit RMS) and combined across threads in FP64: they
// only steer the stop test, which the true residual confirms.
// pslot >= 0 (mixed forms): U was not touched; record alpha_s, the exponent of P_s and its ring slot for
// k_form_u.  pslot < 0 (FP64 form): U was updated; take max|U| for the residual check.
__device__ void fin_update(SolveState* st, const double (&s)[2], int shift, const Geom& g, int pslot) {
  const double rr = ldexp(s[0], -2 * shift), sumR = ldexp(s[1], -shift);
  st->rr = rr;
  st->sumR = sumR;
  st->iter += 1;
  st->zero_guess = 0;
  if (pslot >= 0) {
    const int n = st->n_pend;
    st->pend_alpha[n] = st->alpha;
    st->pend_kp[n] = st->kp;
    st->pend_slot[n] = pslot;
    st->n_pend = n + 1;
  } else {
    st->umax = __longlong_as_double((long long)atomicExch(&st->umax_bits, 0ull));
    plan_residual_check(st, g);
  }
  advance_shift(st, rr, g.N);
  if (!isfinite(rr)) {
    st->status = TPCG_ERR_BREAKDOWN;
    st->done = 1;
    return;
  }
  if (rr <= st->tol2 || st->iter >= st->maxit) st->need_check = 1;
}

// Mixed forms with the deferred U update (TPCG_OPT_DEFER_U): R -= alpha W with W = L P from the exact
// integer stencil of P_int, in a register-window stream (see k_direction_int).  The loads of plane k+1
// (P two planes ahead, the y neighbours and R) are issued before plane k is processed.  U += alpha P is
// not applied: the finalize records it for k_form_u (P_s stays in ring slot pslot until then).
__global__ void __launch_bounds__(TX* TY, 4) k_update_int(Geom g, const int* __restrict__ P, double* __restrict__ R,
                                                          LowPrec lp, SolveState* st, double* partials, int pslot) {
  if (st->done) return;
  const double na0 = st->nah[0], na1 = st->nah[1], na2 = st->nah[2];  // -alpha / h^2 per axis
  const int kp = st->kp;
  const int shift = st->lp_shift;
  const unsigned nx = (unsigned)g.nx, plane = (unsigned)g.nx * (unsigned)g.ny;
  const bool has_z = g.nz > 1;
  const int lane = threadIdx.x;
  float rr = 0.0f, sR = 0.0f;
  for_each_run(g, [&](int bx0, int by0, int k0, int k1) {
    const int x = bx0 + lane, y = by0 + threadIdx.y;
    const bool active = x < g.nx && y < g.ny;
    const unsigned col = (unsigned)y * nx + (unsigned)x;
    const int xgl = ghost_index(x - 1, g.nx, g.bc[0]), xgr = ghost_index(x + 1, g.nx, g.bc[0]);
    const int ygl = ghost_index(y - 1, g.ny, g.bc[1]), ygr = ghost_index(y + 1, g.ny, g.bc[1]);
    const bool own_xl = lane == 0, own_xr = lane == TX - 1 || x == g.nx - 1;  // halo or boundary: load
    auto ld = [&](unsigned k, int xx, int yy) -> int {
      return (xx >= 0 && yy >= 0) ? __ldg(P + k * plane + (unsigned)yy * nx + (unsigned)xx) : 0;
    };
    auto ldz = [&](int kk) -> int {  // P at (x, y, kk), kk possibly a ghost plane
      if (!has_z) return 0;
      const int kz = ghost_index(kk, g.nz, g.bc[2]);
      return (active && kz >= 0) ? __ldg(P + (unsigned)kz * plane + col) : 0;
    };
    struct Plane {
      int c, yl, yr, xl, xr;
      double r;
    };
    auto fetch = [&](int k, int c) {
      Plane f;
      f.c = c;
      f.yl = f.yr = f.xl = f.xr = 0;
      f.r = 0.0;
      if (active) {
        const unsigned kk = (unsigned)k;
        f.yl = ld(kk, x, ygl);
        f.yr = ld(kk, x, ygr);
        if (own_xl) f.xl = ld(kk, xgl, y);
        if (own_xr) f.xr = ld(kk, xgr, y);
        f.r = R[kk * plane + col];
      }
      return f;
    };
    int zl = ldz(k0 - 1);
    const int c0 = active ? __ldg(P + (unsigned)k0 * plane + col) : 0;
    int zr = (k0 + 1 < g.nz) ? (active ? __ldg(P + (unsigned)(k0 + 1) * plane + col) : 0) : ldz(k0 + 1);
    Plane cur = fetch(k0, c0);
    for (int k = k0; k < k1; ++k) {
      // loads for plane k+1 (and P two planes ahead) go out before plane k is processed
      Plane nxt;
      int zr2 = 0;
      if (k + 1 < k1) {
        nxt = fetch(k + 1, zr);
        zr2 = (k + 2 < g.nz) ? (active ? __ldg(P + (unsigned)(k + 2) * plane + col) : 0) : ldz(k + 2);
      }
      const int c = cur.c;
      int xl = __shfl_up_sync(0xffffffffu, c, 1), xr = __shfl_down_sync(0xffffffffu, c, 1);
      if (own_xl) xl = cur.xl;
      if (own_xr) xr = cur.xr;
      const int zlv = has_z ? zl : c, zrv = has_z ? zr : c;
      if (active) {
        const int dx = 2 * c - xl - xr, dy = 2 * c - cur.yl - cur.yr, dz = 2 * c - zlv - zrv;
        double r = cur.r;
        if (g.uniform) {
          r = fma(na0, i32_to_f64_scaled(dx + dy + dz, -kp), r);
        } else {
          r = fma(na0, i32_to_f64_scaled(dx, -kp), r);
          r = fma(na1, i32_to_f64_scaled(dy, -kp), r);
          if (dz) r = fma(na2, i32_to_f64_scaled(dz, -kp), r);
        }
        const unsigned i = (unsigned)k * plane + col;
        R[i] = r;
        const float r32 = f64_to_f32_odd(r, shift);
        store_lp(lp, i, r, r32);
        rr = fmaf(r32, r32, rr);
        sR += r32;
      }
      zl = c;
      zr = zr2;
      if (k + 1 < k1) cur = nxt;
    }
  });
  double acc[2] = {f32_to_f64_int(rr), f32_to_f64_int(sR)};
  grid_reduce<2>(acc, partials, &st->tickets[kTkUpd], gridDim.x, blockIdx.x,
                 [st, shift, g, pslot](const double(&s)[2]) { fin_update(st, s, shift, g, pslot); });
}

// The same update with two adjacent x points per thread (even nx): R moves
// as 16-byte double2, P and its y neighbours as int2, the FP16 copy as one
// packed pair; only the outer x neighbours of a pair come by warp shuffle.
// A warp covers 64 consecutive x of one row.
__global__ void __launch_bounds__(TX* TY, 4) k_update_pair(Geom g, const int* __restrict__ P, double* __restrict__ R,
                                                           LowPrec lp, SolveState* st, double* partials, int pslot) {
  if (st->done) return;
  const double na0 = st->nah[0], na1 = st->nah[1], na2 = st->nah[2];  // -alpha / h^2 per axis
  const int kp = st->kp;
  const int shift = st->lp_shift;
  const unsigned nx = (unsigned)g.nx, plane = (unsigned)g.nx * (unsigned)g.ny;
  const bool has_z = g.nz > 1;
  const int lane = threadIdx.x;
  float rr = 0.0f, sR = 0.0f;
  // instantiated for equal and unequal spacings, so that the per-point code carries one stencil form
  auto sweep = [&](auto uni) {
  constexpr bool kUni = decltype(uni)::value;
  for_each_run<2 * TX>(g, [&](int bx0, int by0, int k0, int k1) {
    const int x = bx0 + 2 * lane, y = by0 + threadIdx.y;  // points (x, y) and (x + 1, y)
    const bool active = x < g.nx && y < g.ny;             // nx even: both points or neither
    const unsigned col = active ? (unsigned)y * nx + (unsigned)x : 0u;
    const int xgl = ghost_index(x - 1, g.nx, g.bc[0]), xgr = ghost_index(x + 2, g.nx, g.bc[0]);
    const int ygl = ghost_index(y - 1, g.ny, g.bc[1]), ygr = ghost_index(y + 1, g.ny, g.bc[1]);
    const bool own_xl = lane == 0, own_xr = lane == TX - 1 || x + 2 >= g.nx;  // halo or boundary
    const unsigned coll = (unsigned)y * nx + (unsigned)max(xgl, 0), colr = (unsigned)y * nx + (unsigned)max(xgr, 0);
    const unsigned colu = (unsigned)max(ygl, 0) * nx + (unsigned)x, cold = (unsigned)max(ygr, 0) * nx + (unsigned)x;
    const bool has_yl = active && ygl >= 0, has_yr = active && ygr >= 0;
    const bool has_xl = active && own_xl && xgl >= 0, has_xr = active && own_xr && xgr >= 0;
    const int2 zero2 = make_int2(0, 0);
    auto ld2 = [&](unsigned i) -> int2 { return __ldg(reinterpret_cast<const int2*>(P + i)); };
    auto ldz = [&](int kk) -> int2 {  // P at (x.., y, kk), kk possibly a ghost plane
      if (!has_z || !active) return zero2;
      const int kz = ghost_index(kk, g.nz, g.bc[2]);
      return kz >= 0 ? ld2((unsigned)kz * plane + col) : zero2;
    };
    struct Plane {
      int2 c, yl, yr;
      int xl, xr;
      double2 r;
    };
    auto fetch = [&](int k, int2 c) {
      Plane f;
      const unsigned base = (unsigned)k * plane;
      f.c = c;
      f.yl = has_yl ? ld2(base + colu) : zero2;
      f.yr = has_yr ? ld2(base + cold) : zero2;
      f.xl = has_xl ? __ldg(P + base + coll) : 0;
      f.xr = has_xr ? __ldg(P + base + colr) : 0;
      f.r = active ? *reinterpret_cast<const double2*>(R + base + col) : make_double2(0.0, 0.0);
      return f;
    };
    int2 zl = ldz(k0 - 1);
    const int2 c0 = active ? ld2((unsigned)k0 * plane + col) : zero2;
    int2 zr = (k0 + 1 < g.nz) ? (active ? ld2((unsigned)(k0 + 1) * plane + col) : zero2) : ldz(k0 + 1);
    Plane cur = fetch(k0, c0);
    for (int k = k0; k < k1; ++k) {
      Plane nxt;
      int2 zr2 = zero2;
      if (k + 1 < k1) {  // loads of plane k+1 (and P two planes ahead) go out before plane k is processed
        nxt = fetch(k + 1, zr);
        zr2 = (k + 2 < g.nz) ? (active ? ld2((unsigned)(k + 2) * plane + col) : zero2) : ldz(k + 2);
      }
      const int2 c = cur.c;
      int xl = __shfl_up_sync(0xffffffffu, c.y, 1), xr = __shfl_down_sync(0xffffffffu, c.x, 1);
      if (own_xl) xl = cur.xl;
      if (own_xr) xr = cur.xr;
      const int2 zlv = has_z ? zl : c, zrv = has_z ? zr : c;
      if (active) {
        const int dx0 = 2 * c.x - xl - c.y, dx1 = 2 * c.y - c.x - xr;
        const int dy0 = 2 * c.x - cur.yl.x - cur.yr.x, dy1 = 2 * c.y - cur.yl.y - cur.yr.y;
        const int dz0 = 2 * c.x - zlv.x - zrv.x, dz1 = 2 * c.y - zlv.y - zrv.y;
        double r0 = cur.r.x, r1 = cur.r.y;
        if constexpr (kUni) {
          r0 = fma(na0, i32_to_f64_scaled(dx0 + dy0 + dz0, -kp), r0);
          r1 = fma(na0, i32_to_f64_scaled(dx1 + dy1 + dz1, -kp), r1);
        } else {
          r0 = fma(na0, i32_to_f64_scaled(dx0, -kp), r0);
          r0 = fma(na1, i32_to_f64_scaled(dy0, -kp), r0);
          if (dz0) r0 = fma(na2, i32_to_f64_scaled(dz0, -kp), r0);
          r1 = fma(na0, i32_to_f64_scaled(dx1, -kp), r1);
          r1 = fma(na1, i32_to_f64_scaled(dy1, -kp), r1);
          if (dz1) r1 = fma(na2, i32_to_f64_scaled(dz1, -kp), r1);
        }
        const unsigned i = (unsigned)k * plane + col;
        *reinterpret_cast<double2*>(R + i) = make_double2(r0, r1);
        const float a32 = f64_to_f32_odd(r0, shift), b32 = f64_to_f32_odd(r1, shift);
        store_lp_pair(lp, i, r0, r1, a32, b32);
        rr = fmaf(a32, a32, fmaf(b32, b32, rr));
        sR += a32 + b32;
      }
      zl = c;
      zr = zr2;
      if (k + 1 < k1) cur = nxt;
    }
  });
  };
  if (g.uniform) sweep(std::true_type{});
  else sweep(std::false_type{});
  double acc[2] = {f32_to_f64_int(rr), f32_to_f64_int(sR)};
  grid_reduce<2>(acc, partials, &st->tickets[kTkUpd], gridDim.x, blockIdx.x,
                 [st, shift, g, pslot](const double(&s)[2]) { fin_update(st, s, shift, g, pslot); });
}

// Mixed forms, U updated in place (the default): U += alpha P and R -= alpha W with W = L P from the
// exact integer stencil of P_int, in a register-window stream (see k_direction_int).  The loads of
// plane k+1 (P two planes ahead, the y neighbours, R and U) are issued before plane k is processed.
// ZG: the first update of a zero initial guess writes U = alpha P.
template <bool ZG>
__global__ void __launch_bounds__(TX* TY, 4) k_update_u_int(Geom g, double* __restrict__ U,
                                                          const int* __restrict__ P, double* __restrict__ R,
                                                          LowPrec lp, SolveState* st, double* partials) {
  if (st->done) return;
  // the solve's buffers come from the state (a captured launch sequence serves every solve of the plan)
  U = st->ups;
  const double alpha = st->alpha;
  const double na0 = st->nah[0], na1 = st->nah[1], na2 = st->nah[2];  // -alpha / h^2 per axis
  const int kp = st->kp;
  const int shift = st->lp_shift;
  const unsigned nx = (unsigned)g.nx, plane = (unsigned)g.nx * (unsigned)g.ny;
  const bool has_z = g.nz > 1;
  const int lane = threadIdx.x;
  float rr = 0.0f, sR = 0.0f;
  unsigned long long um = 0;
  for_each_run(g, [&](int bx0, int by0, int k0, int k1) {
    const int x = bx0 + lane, y = by0 + threadIdx.y;
    const bool active = x < g.nx && y < g.ny;
    const unsigned col = (unsigned)y * nx + (unsigned)x;
    const int xgl = ghost_index(x - 1, g.nx, g.bc[0]), xgr = ghost_index(x + 1, g.nx, g.bc[0]);
    const int ygl = ghost_index(y - 1, g.ny, g.bc[1]), ygr = ghost_index(y + 1, g.ny, g.bc[1]);
    const bool own_xl = lane == 0, own_xr = lane == TX - 1 || x == g.nx - 1;  // halo or boundary: load
    auto ld = [&](unsigned k, int xx, int yy) -> int {
      return (xx >= 0 && yy >= 0) ? __ldg(P + k * plane + (unsigned)yy * nx + (unsigned)xx) : 0;
    };
    auto ldz = [&](int kk) -> int {  // P at (x, y, kk), kk possibly a ghost plane
      if (!has_z) return 0;
      const int kz = ghost_index(kk, g.nz, g.bc[2]);
      return (active && kz >= 0) ? __ldg(P + (unsigned)kz * plane + col) : 0;
    };
    struct Plane {
      int c, yl, yr, xl, xr;
      double r, u;
    };
    auto fetch = [&](int k, int c) {
      Plane f;
      f.c = c;
      f.yl = f.yr = f.xl = f.xr = 0;
      f.r = f.u = 0.0;
      if (active) {
        const unsigned kk = (unsigned)k;
        f.yl = ld(kk, x, ygl);
        f.yr = ld(kk, x, ygr);
        if (own_xl) f.xl = ld(kk, xgl, y);
        if (own_xr) f.xr = ld(kk, xgr, y);
        f.r = R[kk * plane + col];
        if (!ZG) f.u = U[kk * plane + col];
      }
      return f;
    };
    int zl = ldz(k0 - 1);
    const int c0 = active ? __ldg(P + (unsigned)k0 * plane + col) : 0;
    int zr = (k0 + 1 < g.nz) ? (active ? __ldg(P + (unsigned)(k0 + 1) * plane + col) : 0) : ldz(k0 + 1);
    Plane cur = fetch(k0, c0);
    for (int k = k0; k < k1; ++k) {
      // loads for plane k+1 (and P two planes ahead) go out before plane k is processed
      Plane nxt;
      int zr2 = 0;
      if (k + 1 < k1) {
        nxt = fetch(k + 1, zr);
        zr2 = (k + 2 < g.nz) ? (active ? __ldg(P + (unsigned)(k + 2) * plane + col) : 0) : ldz(k + 2);
      }
      const int c = cur.c;
      int xl = __shfl_up_sync(0xffffffffu, c, 1), xr = __shfl_down_sync(0xffffffffu, c, 1);
      if (own_xl) xl = cur.xl;
      if (own_xr) xr = cur.xr;
      const int zlv = has_z ? zl : c, zrv = has_z ? zr : c;
      if (active) {
        const int dx = 2 * c - xl - xr, dy = 2 * c - cur.yl - cur.yr, dz = 2 * c - zlv - zrv;
        double r = cur.r;
        if (g.uniform) {
          r = fma(na0, i32_to_f64_scaled(dx + dy + dz, -kp), r);
        } else {
          r = fma(na0, i32_to_f64_scaled(dx, -kp), r);
          r = fma(na1, i32_to_f64_scaled(dy, -kp), r);
          if (dz) r = fma(na2, i32_to_f64_scaled(dz, -kp), r);
        }
        const unsigned i = (unsigned)k * plane + col;
        R[i] = r;
        const float r32 = f64_to_f32_odd(r, shift);
        store_lp(lp, i, r, r32);
        rr = fmaf(r32, r32, rr);
        sR += r32;
        const double pv = i32_to_f64_scaled(c, -kp);
        const double u = ZG ? alpha * pv : fma(alpha, pv, cur.u);
        U[i] = u;
        const unsigned long long ub = mag_key(u);
        um = ub > um ? ub : um;
      }
      zl = c;
      zr = zr2;
      if (k + 1 < k1) cur = nxt;
    }
  });
  double acc[2] = {f32_to_f64_int(rr), f32_to_f64_int(sR)};
  fold_umax(st, um);
  grid_reduce<2>(acc, partials, &st->tickets[kTkUpd], gridDim.x, blockIdx.x,
                 [st, shift, g](const double(&s)[2]) { fin_update(st, s, shift, g, -1); });
}

// The same in-place update with two adjacent x points per thread (even nx): R and U move
// as 16-byte double2, P and its y neighbours as int2, the FP16 copy as one
// packed pair; only the outer x neighbours of a pair come by warp shuffle.
// A warp covers 64 consecutive x of one row.
template <bool ZG>
__global__ void __launch_bounds__(TX* TY, 4) k_update_u_pair(Geom g, double* __restrict__ U,
                                                           const int* __restrict__ P, double* __restrict__ R,
                                                           LowPrec lp, SolveState* st, double* partials) {
  if (st->done) return;
  // the solve's buffers come from the state (a captured launch sequence serves every solve of the plan)
  U = st->ups;
  const double alpha = st->alpha;
  const double na0 = st->nah[0], na1 = st->nah[1], na2 = st->nah[2];  // -alpha / h^2 per axis
  const int kp = st->kp;
  const int shift = st->lp_shift;
  const unsigned nx = (unsigned)g.nx, plane = (unsigned)g.nx * (unsigned)g.ny;
  const bool has_z = g.nz > 1;
  const int lane = threadIdx.x;
  float rr = 0.0f, sR = 0.0f;
  unsigned long long um = 0;
  // instantiated for equal and unequal spacings, so that the per-point code carries one stencil form
  auto sweep = [&](auto uni) {
  constexpr bool kUni = decltype(uni)::value;
  for_each_run<2 * TX>(g, [&](int bx0, int by0, int k0, int k1) {
    const int x = bx0 + 2 * lane, y = by0 + threadIdx.y;  // points (x, y) and (x + 1, y)
    const bool active = x < g.nx && y < g.ny;             // nx even: both points or neither
    const unsigned col = active ? (unsigned)y * nx + (unsigned)x : 0u;
    const int xgl = ghost_index(x - 1, g.nx, g.bc[0]), xgr = ghost_index(x + 2, g.nx, g.bc[0]);
    const int ygl = ghost_index(y - 1, g.ny, g.bc[1]), ygr = ghost_index(y + 1, g.ny, g.bc[1]);
    const bool own_xl = lane == 0, own_xr = lane == TX - 1 || x + 2 >= g.nx;  // halo or boundary
    const unsigned coll = (unsigned)y * nx + (unsigned)max(xgl, 0), colr = (unsigned)y * nx + (unsigned)max(xgr, 0);
    const unsigned colu = (unsigned)max(ygl, 0) * nx + (unsigned)x, cold = (unsigned)max(ygr, 0) * nx + (unsigned)x;
    const bool has_yl = active && ygl >= 0, has_yr = active && ygr >= 0;
    const bool has_xl = active && own_xl && xgl >= 0, has_xr = active && own_xr && xgr >= 0;
    const int2 zero2 = make_int2(0, 0);
    auto ld2 = [&](unsigned i) -> int2 { return __ldg(reinterpret_cast<const int2*>(P + i)); };
    auto ldz = [&](int kk) -> int2 {  // P at (x.., y, kk), kk possibly a ghost plane
      if (!has_z || !active) return zero2;
      const int kz = ghost_index(kk, g.nz, g.bc[2]);
      return kz >= 0 ? ld2((unsigned)kz * plane + col) : zero2;
    };
    struct Plane {
      int2 c, yl, yr;
      int xl, xr;
      double2 r, u;
    };
    auto fetch = [&](int k, int2 c) {
      Plane f;
      const unsigned base = (unsigned)k * plane;
      f.c = c;
      f.yl = has_yl ? ld2(base + colu) : zero2;
      f.yr = has_yr ? ld2(base + cold) : zero2;
      f.xl = has_xl ? __ldg(P + base + coll) : 0;
      f.xr = has_xr ? __ldg(P + base + colr) : 0;
      f.r = active ? *reinterpret_cast<const double2*>(R + base + col) : make_double2(0.0, 0.0);
      f.u = (active && !ZG) ? *reinterpret_cast<const double2*>(U + base + col) : make_double2(0.0, 0.0);
      return f;
    };
    int2 zl = ldz(k0 - 1);
    const int2 c0 = active ? ld2((unsigned)k0 * plane + col) : zero2;
    int2 zr = (k0 + 1 < g.nz) ? (active ? ld2((unsigned)(k0 + 1) * plane + col) : zero2) : ldz(k0 + 1);
    Plane cur = fetch(k0, c0);
    for (int k = k0; k < k1; ++k) {
      Plane nxt;
      int2 zr2 = zero2;
      if (k + 1 < k1) {  // loads of plane k+1 (and P two planes ahead) go out before plane k is processed
        nxt = fetch(k + 1, zr);
        zr2 = (k + 2 < g.nz) ? (active ? ld2((unsigned)(k + 2) * plane + col) : zero2) : ldz(k + 2);
      }
      const int2 c = cur.c;
      int xl = __shfl_up_sync(0xffffffffu, c.y, 1), xr = __shfl_down_sync(0xffffffffu, c.x, 1);
      if (own_xl) xl = cur.xl;
      if (own_xr) xr = cur.xr;
      const int2 zlv = has_z ? zl : c, zrv = has_z ? zr : c;
      if (active) {
        const int dx0 = 2 * c.x - xl - c.y, dx1 = 2 * c.y - c.x - xr;
        const int dy0 = 2 * c.x - cur.yl.x - cur.yr.x, dy1 = 2 * c.y - cur.yl.y - cur.yr.y;
        const int dz0 = 2 * c.x - zlv.x - zrv.x, dz1 = 2 * c.y - zlv.y - zrv.y;
        double r0 = cur.r.x, r1 = cur.r.y;
        if constexpr (kUni) {
          r0 = fma(na0, i32_to_f64_scaled(dx0 + dy0 + dz0, -kp), r0);
          r1 = fma(na0, i32_to_f64_scaled(dx1 + dy1 + dz1, -kp), r1);
        } else {
          r0 = fma(na0, i32_to_f64_scaled(dx0, -kp), r0);
          r0 = fma(na1, i32_to_f64_scaled(dy0, -kp), r0);
          if (dz0) r0 = fma(na2, i32_to_f64_scaled(dz0, -kp), r0);
          r1 = fma(na0, i32_to_f64_scaled(dx1, -kp), r1);
          r1 = fma(na1, i32_to_f64_scaled(dy1, -kp), r1);
          if (dz1) r1 = fma(na2, i32_to_f64_scaled(dz1, -kp), r1);
        }
        const unsigned i = (unsigned)k * plane + col;
        *reinterpret_cast<double2*>(R + i) = make_double2(r0, r1);
        const float a32 = f64_to_f32_odd(r0, shift), b32 = f64_to_f32_odd(r1, shift);
        store_lp_pair(lp, i, r0, r1, a32, b32);
        rr = fmaf(a32, a32, fmaf(b32, b32, rr));
        sR += a32 + b32;
        const double p0 = i32_to_f64_scaled(c.x, -kp), p1 = i32_to_f64_scaled(c.y, -kp);
        const double u0 = ZG ? alpha * p0 : fma(alpha, p0, cur.u.x);
        const double u1 = ZG ? alpha * p1 : fma(alpha, p1, cur.u.y);
        *reinterpret_cast<double2*>(U + i) = make_double2(u0, u1);
        const unsigned long long k0b = mag_key(u0), k1b = mag_key(u1);
        const unsigned long long kb = k0b > k1b ? k0b : k1b;
        um = kb > um ? kb : um;
      }
      zl = c;
      zr = zr2;
      if (k + 1 < k1) cur = nxt;
    }
  });
  };
  if (g.uniform) sweep(std::true_type{});
  else sweep(std::false_type{});
  double acc[2] = {f32_to_f64_int(rr), f32_to_f64_int(sR)};
  fold_umax(st, um);
  grid_reduce<2>(acc, partials, &st->tickets[kTkUpd], gridDim.x, blockIdx.x,
                 [st, shift, g](const double(&s)[2]) { fin_update(st, s, shift, g, -1); });
}

// FP64 form: P and W = L P are stored by the direction kernel.
__global__ void __launch_bounds__(256) k_update(Geom g, double* __restrict__ U, const double* __restrict__ P,
                                                const double* __restrict__ W, double* __restrict__ R, LowPrec lp,
                                                SolveState* st, double* partials) {
  const long long N = g.N;
  if (st->done) return;
  // the solve's buffers come from the state (a captured launch sequence serves every solve of the plan)
  U = st->ups;
  const double alpha = st->alpha;
  const double nalpha = -alpha;
  const int zg = st->zero_guess;
  const int shift = st->lp_shift;
  float a0 = 0.0f, a1 = 0.0f;
  unsigned long long um = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    const double p = __ldg(P + i);
    const double u = zg ? alpha * p : fma(alpha, p, U[i]);
    U[i] = u;
    const unsigned long long ub = mag_key(u);
    um = ub > um ? ub : um;
    const double r = fma(nalpha, __ldg(W + i), R[i]);
    R[i] = r;
    const float r32 = f64_to_f32_odd(r, shift);
    store_lp(lp, i, r, r32);
    a0 = fmaf(r32, r32, a0);
    a1 += r32;
  }
  fold_umax(st, um);
  double acc[2] = {f32_to_f64_int(a0), f32_to_f64_int(a1)};
  grid_reduce<2>(acc, partials, &st->tickets[kTkUpd], gridDim.x, blockIdx.x,
                 [st, shift, g](const double(&s)[2]) { fin_update(st, s, shift, g, -1); });
}

// ------------------------------------------------------------------ streaming kernels
// R = eta_hat (zero initial guess: U_0 = 0 in Algorithm 1); ||eta_hat||^2 in
// FP64 (it scales the tolerance and is reported), sum(R) in FP32 from
// R * 2^lp_shift.
__global__ void __launch_bounds__(256) k_init_zero(long long N, const double* __restrict__ eta,
                                                   double* __restrict__ R, LowPrec lp, SolveState* st,
                                                   double* partials) {
  // the solve's buffers come from the state (a captured launch sequence serves every solve of the plan)
  eta = st->eta;
  const double mean = st->mean_eta;
  const int shift = st->lp_shift;
  double e2 = 0.0;
  float a1 = 0.0f;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    const double r = __ldg(eta + i) - mean;
    R[i] = r;
    const float r32 = f64_to_f32_odd(r, shift);
    store_lp(lp, i, r, r32);
    e2 = fma(r, r, e2);
    a1 += r32;
  }
  double acc[2] = {e2, f32_to_f64_int(a1)};
  grid_reduce<2>(acc, partials, &st->tickets[kTkInit], gridDim.x, blockIdx.x, [st, N, shift](const double(&s)[2]) {
    const double v[3] = {s[0], ldexp(s[1], -shift), s[0]};
    fin_init(st, v, N);
  });
}

// sum(eta) and sum(eta^2): the mean removed by eq. (centering) when the
// operator is singular, and the exponent of the first low-precision copy;
// with a given initial guess also max|U_0| for the fixed-point residual.
__global__ void __launch_bounds__(256) k_eta_sum(Geom g, const double* __restrict__ eta,
                                                 const double* __restrict__ U0, SolveState* st, double* partials) {
  // the solve's buffers come from the state (a captured launch sequence serves every solve of the plan)
  eta = st->eta;
  if (U0) U0 = st->ups;  // (NULL: zero initial guess)
  const long long N = g.N;
  double acc[2] = {0.0, 0.0};
  unsigned long long um = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    const double e = __ldg(eta + i);
    acc[0] += e;
    acc[1] = fma(e, e, acc[1]);
    if (U0) {
      const unsigned long long ub = mag_key(__ldg(U0 + i));
      um = ub > um ? ub : um;
    }
  }
  fold_umax(st, um);
  grid_reduce<2>(acc, partials, &st->tickets[kTkEta], gridDim.x, blockIdx.x, [st, N, g](const double(&s)[2]) {
    const double mean = st->singular ? s[0] / (double)N : 0.0;
    st->mean_eta = mean;
    const double n2 = s[1] - mean * s[0];
    st->eta_norm2 = n2 > 0.0 ? n2 : s[1];  // estimate; the initial residual kernel sets the exact value
    st->lp_shift = lp_shift_for(n2 > 0.0 ? n2 : s[1], N);
    st->umax = __longlong_as_double((long long)atomicExch(&st->umax_bits, 0ull));
    plan_residual_check(st, g);
  });
}

// Deferred U update of the mixed forms (Algorithm 1: U_{s+1} = U_s + alpha_s P_s).
// The update kernel records alpha_s, the exponent of P_s = 2^-kp_s P_int,s and
// its ring slot; this kernel applies the recorded updates in iteration order,
// one FP64 FMA each -- the operations, in the order, of updating U every
// iteration -- and takes max|U| for the fixed-point residual check.  It runs
// when a true-residual check is due, when the ring of directions is about to
// wrap, and (force) before the host reads an iterate.  Every block takes the
// same decision from the state, which only the last block's finalize changes.
// PAIR: two adjacent points per thread (N even, U 16-byte aligned).
template <bool PAIR>
__global__ void __launch_bounds__(256) k_form_u(Geom g, double* __restrict__ U, const int* __restrict__ Pring,
                                                unsigned long long pstride, SolveState* st, double* partials,
                                                int force) {
  const int n = st->n_pend;
  if (n == 0 || (!force && (st->done || (!st->need_check && n < kPRing - 1)))) return;
  // the solve's buffers come from the state (a captured launch sequence serves every solve of the plan)
  U = st->ups;
  const bool valid = st->u_valid != 0;
  double al[kPRing - 1];
  int kpn[kPRing - 1];
  const int* pp[kPRing - 1];
#pragma unroll
  for (int k = 0; k < kPRing - 1; ++k) {
    const bool on = k < n;
    al[k] = on ? st->pend_alpha[k] : 0.0;
    kpn[k] = on ? -st->pend_kp[k] : 0;
    pp[k] = Pring + (on ? (unsigned long long)st->pend_slot[k] * pstride : 0ull);
  }
  unsigned long long um = 0;
  const unsigned long long N = (unsigned long long)g.N;
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  if (PAIR) {
    for (unsigned long long t = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; t < N / 2; t += stride) {
      const int2 q0 = __ldg(reinterpret_cast<const int2*>(pp[0]) + t);
      double u0, u1;
      if (valid) {
        const double2 u = reinterpret_cast<const double2*>(U)[t];
        u0 = fma(al[0], i32_to_f64_scaled(q0.x, kpn[0]), u.x);
        u1 = fma(al[0], i32_to_f64_scaled(q0.y, kpn[0]), u.y);
      } else {  // zero initial guess: the first update writes U = alpha_0 P_0
        u0 = al[0] * i32_to_f64_scaled(q0.x, kpn[0]);
        u1 = al[0] * i32_to_f64_scaled(q0.y, kpn[0]);
      }
#pragma unroll
      for (int k = 1; k < kPRing - 1; ++k) {
        if (k < n) {
          const int2 q = __ldg(reinterpret_cast<const int2*>(pp[k]) + t);
          u0 = fma(al[k], i32_to_f64_scaled(q.x, kpn[k]), u0);
          u1 = fma(al[k], i32_to_f64_scaled(q.y, kpn[k]), u1);
        }
      }
      reinterpret_cast<double2*>(U)[t] = make_double2(u0, u1);
      const unsigned long long a = mag_key(u0), b = mag_key(u1);
      const unsigned long long m = a > b ? a : b;
      um = m > um ? m : um;
    }
  } else {
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < N; i += stride) {
      const int q0 = __ldg(pp[0] + i);
      double u = valid ? fma(al[0], i32_to_f64_scaled(q0, kpn[0]), U[i]) : al[0] * i32_to_f64_scaled(q0, kpn[0]);
#pragma unroll
      for (int k = 1; k < kPRing - 1; ++k)
        if (k < n) u = fma(al[k], i32_to_f64_scaled(__ldg(pp[k] + i), kpn[k]), u);
      U[i] = u;
      const unsigned long long m = mag_key(u);
      um = m > um ? m : um;
    }
  }
  fold_umax(st, um);
  double acc[1] = {0.0};
  grid_reduce<1>(acc, partials, &st->tickets[kTkForm], gridDim.x, blockIdx.x, [st, g](const double(&)[1]) {
    st->n_pend = 0;
    st->u_valid = 1;
    st->umax = __longlong_as_double((long long)atomicExch(&st->umax_bits, 0ull));
    plan_residual_check(st, g);
  });
}

// k_init_zero and k_eta_sum with two adjacent points per thread (N even and
// below 2^32; nx even when there is a low-precision copy, so a pair never
// straddles a padded row): 16-byte loads and stores and 32-bit indices.
__global__ void __launch_bounds__(256) k_init_zero2(unsigned npair, long long N, const double* __restrict__ eta,
                                                    double* __restrict__ R, LowPrec lp, SolveState* st,
                                                    double* partials) {
  // the solve's buffers come from the state (a captured launch sequence serves every solve of the plan)
  eta = st->eta;
  const double mean = st->mean_eta;
  const int shift = st->lp_shift;
  double e2 = 0.0;
  float a1 = 0.0f;
  const unsigned stride = gridDim.x * blockDim.x;
  for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < npair; t += stride) {
    const double2 e = __ldg(reinterpret_cast<const double2*>(eta) + t);
    const double r0 = e.x - mean, r1 = e.y - mean;
    reinterpret_cast<double2*>(R)[t] = make_double2(r0, r1);
    const float a32 = f64_to_f32_odd(r0, shift), b32 = f64_to_f32_odd(r1, shift);
    store_lp_pair(lp, 2ll * t, r0, r1, a32, b32);
    e2 = fma(r0, r0, fma(r1, r1, e2));
    a1 += a32 + b32;
  }
  double acc[2] = {e2, f32_to_f64_int(a1)};
  grid_reduce<2>(acc, partials, &st->tickets[kTkInit], gridDim.x, blockIdx.x, [st, N, shift](const double(&s)[2]) {
    const double v[3] = {s[0], ldexp(s[1], -shift), s[0]};
    fin_init(st, v, N);
  });
}

__global__ void __launch_bounds__(256) k_eta_sum2(Geom g, unsigned npair, const double* __restrict__ eta,
                                                  const double* __restrict__ U0, SolveState* st, double* partials) {
  // the solve's buffers come from the state (a captured launch sequence serves every solve of the plan)
  eta = st->eta;
  if (U0) U0 = st->ups;  // (NULL: zero initial guess)
  const long long N = g.N;
  double acc[2] = {0.0, 0.0};
  unsigned long long um = 0;
  const unsigned stride = gridDim.x * blockDim.x;
  for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < npair; t += stride) {
    const double2 e = __ldg(reinterpret_cast<const double2*>(eta) + t);
    acc[0] += e.x;
    acc[0] += e.y;
    acc[1] = fma(e.y, e.y, fma(e.x, e.x, acc[1]));
    if (U0) {
      const double2 u = __ldg(reinterpret_cast<const double2*>(U0) + t);
      const unsigned long long a = mag_key(u.x), b = mag_key(u.y);
      const unsigned long long ub = a > b ? a : b;
      um = ub > um ? ub : um;
    }
  }
  fold_umax(st, um);
  grid_reduce<2>(acc, partials, &st->tickets[kTkEta], gridDim.x, blockIdx.x, [st, N, g](const double(&s)[2]) {
    const double mean = st->singular ? s[0] / (double)N : 0.0;
    st->mean_eta = mean;
    const double n2 = s[1] - mean * s[0];
    st->eta_norm2 = n2 > 0.0 ? n2 : s[1];  // estimate; the initial residual kernel sets the exact value
    st->lp_shift = lp_shift_for(n2 > 0.0 ? n2 : s[1], N);
    st->umax = __longlong_as_double((long long)atomicExch(&st->umax_bits, 0ull));
    plan_residual_check(st, g);
  });
}

// ||r||^2 -> exponent of the low-precision copy (tpcg_precond_apply).
__global__ void __launch_bounds__(256) k_norm_shift(long long N, const double* __restrict__ r, SolveState* st,
                                                    double* partials) {
  double acc[1] = {0.0};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    const double v = __ldg(r + i);
    acc[0] = fma(v, v, acc[0]);
  }
  grid_reduce<1>(acc, partials, &st->tickets[kTkMisc], gridDim.x, blockIdx.x,
                 [st, N](const double(&s)[1]) { st->lp_shift = lp_shift_for(s[0], N); });
}

// U -= sum(U)/N: return the zero-mean (minimum-norm) representative.  With
// iter_lo >= 0 only when the solve converged in an iteration after iter_lo:
// launched behind each chunk of iterations, it centres U in the chunk where
// the stop test succeeded (every block takes the same decision: done_iter is
// set once) and saves the host a round trip.
__global__ void __launch_bounds__(256) k_center_u(long long N, double* __restrict__ U, const SolveState* st,
                                                  int iter_lo) {
  if (iter_lo >= 0 && !(st->done == 1 && st->status == TPCG_OK && st->done_iter > iter_lo)) return;
  // the solve's buffers come from the state (a captured launch sequence serves every solve of the plan)
  U = st->ups;
  const double m = st->sumU / (double)N;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x)
    U[i] -= m;
}

__global__ void k_zero(long long N, double* __restrict__ U) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x)
    U[i] = 0.0;
}

// Low-precision copy of an FP64 field with the state's current exponent
// (tpcg_precond_apply, and the warm-started FP16 form after its first residual).
__global__ void __launch_bounds__(256) k_to_lp(long long N, const double* __restrict__ r, LowPrec lp,
                                               SolveState* st) {
  const int shift = st->lp_shift;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x)
  {
    const double v = __ldg(r + i);
    store_lp(lp, i, v, f64_to_f32_odd(v, shift));
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) st->lp_shift_applied = shift;
}

// FP32 -> FP64 copy (Z of the mixed forms, for tpcg_precond_apply).
__global__ void __launch_bounds__(256) k_f32_to_f64(long long N, const float* __restrict__ a, double* __restrict__ b) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x)
    b[i] = f32_to_f64_int(__ldg(a + i));
}

// The mixed forms' fixed-point direction P = P_int * 2^-kp as FP64 (exact).
__global__ void __launch_bounds__(256) k_fixed_to_f64(long long N, const int* __restrict__ a, int kp,
                                                      double* __restrict__ b) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x)
    b[i] = i32_to_f64_scaled(__ldg(a + i), -kp);
}

// Sec. 3.4.2: fold constant boundary data into the right-hand side.  bval[2m]
// at the start face of axis m, bval[2m+1] at the end face; Dirichlet adds
// u/h^2 to the boundary layer, Neumann adds e/h (e: outward derivative).
__global__ void k_rhs_add_bc(Geom g, double* __restrict__ eta, double b0, double b1, double b2, double b3, double b4,
                             double b5) {
  const double bv[6] = {b0, b1, b2, b3, b4, b5};
  const unsigned plane = (unsigned)g.nx * (unsigned)g.ny;  // N <= 2^31: 32-bit index arithmetic
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < g.N; i += (long long)gridDim.x * blockDim.x) {
    const unsigned ui = (unsigned)i;
    const int k = (int)(ui / plane);
    const unsigned rem = ui - (unsigned)k * plane;
    const int y = (int)(rem / (unsigned)g.nx), x = (int)(rem - (unsigned)y * (unsigned)g.nx);
    const int pos[3] = {x, y, k};
    const int len[3] = {g.nx, g.ny, g.nz};
    double add = 0.0;
    for (int m = 0; m < 3; ++m) {
      if (len[m] == 1 || g.bc[m] == kBcP) continue;
      const double ih2 = g.ih2[m];
      const double ih = sqrt(ih2);
      const int bc = g.bc[m];
      const bool startD = (bc == kBcD || bc == kBcDN), endD = (bc == kBcD || bc == kBcND);
      if (pos[m] == 0) add += startD ? bv[2 * m] * ih2 : bv[2 * m] * ih;
      if (pos[m] == len[m] - 1) add += endD ? bv[2 * m + 1] * ih2 : bv[2 * m + 1] * ih;
    }
    if (add != 0.0) eta[i] += add;
  }
}


// ------------------------------------------------------------------ comparator preconditioners
// Jacobi(p, omega), Algorithms 2/3 (Sec. 4.3.1): X_0 = 0, X_j = X_{j-1} + (R - L X_{j-1}) / (omega d)
// -- the same iteration as F_j = R - O_omega X_{j-1}, X_j = F_j / (omega d), with O_omega = L - omega D.
// d depends only on whether a point is the first, an interior or the last point of each axis.
struct JacobiTable {
  double invd[27];
};

__device__ __forceinline__ double jacobi_invd(const JacobiTable& t, const Geom& g, unsigned i) {
  const unsigned plane = (unsigned)g.nx * (unsigned)g.ny;
  const int k = (int)(i / plane);
  const unsigned rem = i - (unsigned)k * plane;
  const int y = (int)(rem / (unsigned)g.nx), x = (int)(rem - (unsigned)y * (unsigned)g.nx);
  auto cls = [](int pos, int len) { return len == 1 ? 1 : (pos == 0 ? 0 : (pos == len - 1 ? 2 : 1)); };
  return t.invd[cls(x, g.nx) + 3 * cls(y, g.ny) + 9 * cls(k, g.nz)];
}

__global__ void __launch_bounds__(256) k_jacobi_first(Geom g, const double* __restrict__ R, double* __restrict__ X,
                                                      JacobiTable t) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < g.N; i += (long long)gridDim.x * blockDim.x)
    X[i] = __ldg(R + i) * jacobi_invd(t, g, (unsigned)i);
}

struct OpJacobi {
  const double* __restrict__ R;
  double* __restrict__ Xnew;
  JacobiTable t;
  Geom g;
  __device__ __forceinline__ void operator()(long long i, double c, double w, double (&)[1]) {
    Xnew[i] = fma(__ldg(R + i) - w, jacobi_invd(t, g, (unsigned)i), c);
  }
};

__global__ void __launch_bounds__(TX* TY) k_jacobi_sweep(Geom g, int zchunk, const double* __restrict__ Xold,
                                                         double* __restrict__ Xnew, const double* __restrict__ R,
                                                         JacobiTable t) {
  FieldPlain f{Xold};
  OpJacobi op{R, Xnew, t, g};
  stencil_sweep<0>(g, zchunk, f, op, nullptr, nullptr, NoFin{});
}

// rho = <R, Z> and sum(Z) in FP64 (comparators); Z = R first when copy (M = I).
__global__ void __launch_bounds__(256) k_dot_rz(long long N, const double* __restrict__ R, double* __restrict__ Z,
                                                int copy, SolveState* st, double* partials) {
  double acc[2] = {0.0, 0.0};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    const double r = __ldg(R + i);
    const double z = copy ? r : Z[i];
    if (copy) Z[i] = r;
    acc[0] = fma(r, z, acc[0]);
    acc[1] += z;
  }
  if (!st) return;
  grid_reduce<2>(acc, partials, &st->tickets[kTkPrec], gridDim.x, blockIdx.x,
                 [st, N](const double(&s)[2]) { fin_precond(st, N, s); });
}

// ------------------------------------------------------------------ electric field
// epsilon = -grad(ups) (Sec. 2; the field of the computed potential) by central
// differences -(u_{i+1} - u_{i-1}) / (2 h).  The neighbour across a face is the
// ghost value of the Laplacian's boundary condition (eq. lap1d) with the face
// data of Sec. 3.4.2: periodic faces wrap, a Dirichlet face holds u_B, a Neumann
// face holds u_boundary + h e_B (e_B the outward normal derivative).
struct FaceData {
  double v[6];      // face data, start and end face per axis (0: homogeneous)
  double h[3];      // spacing per axis
  double inv2h[3];  // 1 / (2 h)
};

__global__ void __launch_bounds__(256) k_efield(Geom g, const double* __restrict__ U, FaceData fd,
                                                double* __restrict__ ex, double* __restrict__ ey,
                                                double* __restrict__ ez) {
  const unsigned plane = (unsigned)g.nx * (unsigned)g.ny;  // N <= 2^31: 32-bit index arithmetic
  const int naxes = g.nz > 1 ? 3 : 2;
  for (long long ii = blockIdx.x * (long long)blockDim.x + threadIdx.x; ii < g.N;
       ii += (long long)gridDim.x * blockDim.x) {
    const unsigned i = (unsigned)ii;
    const int k = (int)(i / plane);
    const unsigned rem = i - (unsigned)k * plane;
    const int y = (int)(rem / (unsigned)g.nx), x = (int)(rem - (unsigned)y * (unsigned)g.nx);
    const int pos[3] = {x, y, k}, len[3] = {g.nx, g.ny, g.nz};
    const unsigned stride[3] = {1u, (unsigned)g.nx, plane};
    const double u0 = __ldg(U + i);
    for (int m = 0; m < naxes; ++m) {
      const int bc = g.bc[m];
      const bool startD = bc == kBcD || bc == kBcDN, endD = bc == kBcD || bc == kBcND;
      double lo, hi;
      if (pos[m] > 0) lo = __ldg(U + i - stride[m]);
      else if (bc == kBcP) lo = __ldg(U + i + (unsigned)(len[m] - 1) * stride[m]);
      else lo = startD ? fd.v[2 * m] : fma(fd.h[m], fd.v[2 * m], u0);
      if (pos[m] < len[m] - 1) hi = __ldg(U + i + stride[m]);
      else if (bc == kBcP) hi = __ldg(U + i - (unsigned)(len[m] - 1) * stride[m]);
      else hi = endD ? fd.v[2 * m + 1] : fma(fd.h[m], fd.v[2 * m + 1], u0);
      double* out = m == 0 ? ex : (m == 1 ? ey : ez);
      out[i] = (lo - hi) * fd.inv2h[m];
    }
  }
}

// ------------------------------------------------------------------ host launchers
void launch_apply_laplacian(const tpcg_plan* p, const Geom& g, const double* x, double* w) {
  LaunchScope ls(p, kKApply);
  k_apply_laplacian<<<p->st_grid, p->st_block, 0, p->stream>>>(g, p->st_zchunk, x, w);
}
// Persistent grids of the fixed-point sweeps: every SM holds as many blocks as
// the kernel's resources allow (at most 8), and every block takes at least
// sweep_grain (tile, plane) pairs; the grid-stride kernels at most 8 blocks per
// SM of at least 256 * sweep_grain points.  A small grid thus leaves SMs to the
// kernels of other plans.
int setup_fx_grids(tpcg_plan* p) {
  const long long grain = p->sweep_grain;
  p->stream_blocks = (int)std::max(1LL, std::min<long long>((p->N + 256 * grain - 1) / (256 * grain),
                                                           (long long)p->num_sms * 8));
  const bool pair = p->nx % 2 == 0;  // direction and update take two x points per thread
  const bool quad = p->nx % 4 == 0;  // direction takes four
  const void* fns[kFxCount] = {quad ? (const void*)k_direction_quad
                                    : (pair ? (const void*)k_direction_pair : (const void*)k_direction_int),
                               pair ? (const void*)k_update_pair : (const void*)k_update_int,
                               (const void*)k_residual_fx<false>, (const void*)k_residual_fx<true>};
  for (int i = 0; i < kFxCount; ++i) {
    const int tw = (i == kFxDir && quad) ? 4 * TX : (((i == kFxUpd || i == kFxDir) && pair) ? 2 * TX : TX);
    const long long T = (long long)((p->nx + tw - 1) / tw) * ((p->ny + TY - 1) / TY) * p->nz;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fns[i], TX * TY, 0) != cudaSuccess) return -1;
    per_sm = std::max(1, std::min(per_sm, 8));
    p->fx_blocks[i] = (int)std::max(1LL, std::min<long long>((T + grain - 1) / grain, (long long)p->num_sms * per_sm));
  }
  return 0;
}
LowPrec lowprec(const tpcg_plan* p) {
  return LowPrec{p->d_Rlp, p->lp_kind, p->pitch16[0], p->nx, (long long)p->lp_plane};
}

// The caller's arrays are device pointers to doubles: only 8-byte alignment is guaranteed, so the
// kernels that move them as 16-byte pairs run only when the pointers allow it.
static bool aligned16(const void* a) { return ((uintptr_t)a & 15) == 0; }
// two points per thread when the point count is even and below 2^32, a pair never straddles a padded
// row of the low-precision copy and the caller's arrays a, b (may be NULL) allow 16-byte accesses
static bool pairs_ok(const tpcg_plan* p, const Geom& g, const void* a, const void* b) {
  return g.N % 2 == 0 && g.N < (1ll << 32) && (p->d_Rlp == nullptr || g.nx % 2 == 0) && aligned16(a) && aligned16(b);
}
void launch_init_residual(const tpcg_plan* p, const Geom& g, const double* eta, const double* U, bool zero_guess) {
  LaunchScope ls(p, kKInit);
  if (zero_guess && pairs_ok(p, g, eta, nullptr))
    k_init_zero2<<<p->stream_blocks, 256, 0, p->stream>>>((unsigned)(g.N / 2), g.N, eta, p->d_R, lowprec(p),
                                                          p->d_state, p->d_partials);
  else if (zero_guess)
    k_init_zero<<<p->stream_blocks, 256, 0, p->stream>>>(g.N, eta, p->d_R, lowprec(p), p->d_state, p->d_partials);
  else
    k_residual_fx<true><<<p->fx_blocks[kFxInit], p->st_block, 0, p->stream>>>(g, eta, U, p->d_R, lowprec(p),
                                                                               p->d_state, p->d_partials, 0);
}
void launch_eta_sum(const tpcg_plan* p, const Geom& g, const double* eta, const double* U0) {
  LaunchScope ls(p, kKEtaSum);
  if (pairs_ok(p, g, eta, U0))
    k_eta_sum2<<<p->stream_blocks, 256, 0, p->stream>>>(g, (unsigned)(g.N / 2), eta, U0, p->d_state, p->d_partials);
  else
    k_eta_sum<<<p->stream_blocks, 256, 0, p->stream>>>(g, eta, U0, p->d_state, p->d_partials);
}
void launch_norm_shift(const tpcg_plan* p, const Geom& g, const double* r) {
  LaunchScope ls(p, kKConvert);
  k_norm_shift<<<p->stream_blocks, 256, 0, p->stream>>>(g.N, r, p->d_state, p->d_partials);
}
// FP64 form: P_k is written to d_P[k & 1], P_{k-1} read from the other buffer.  Mixed forms: P_k goes to
// ring slot k % p_slots (with TPCG_OPT_DEFER_U, kept there until k_form_u has applied alpha_k P_k to U).
void launch_direction(const tpcg_plan* p, const Geom& g, int k) {
  LaunchScope ls(p, kKDirection);
  if (p->prec == TPCG_FP64) {
    k_direction<<<p->st_grid, p->st_block, 0, p->stream>>>(
        g, p->st_zchunk, (const double*)p->d_Z, (const double*)p->d_P[(k + 1) & 1], (double*)p->d_P[k & 1], p->d_W,
        p->d_state, p->d_partials);
    return;
  }
  const int ns = p->p_slots;
  const int* Pold = (const int*)p->d_P[(k + ns - 1) % ns];
  int* Pnew = (int*)p->d_P[k % ns];
  if (g.nx % 4 == 0)
    k_direction_quad<<<p->fx_blocks[kFxDir], p->st_block, 0, p->stream>>>(g, (const float*)p->d_Z, Pold, Pnew,
                                                                           p->d_state, p->d_partials);
  else if (g.nx % 2 == 0)
    k_direction_pair<<<p->fx_blocks[kFxDir], p->st_block, 0, p->stream>>>(g, (const float*)p->d_Z, Pold, Pnew,
                                                                           p->d_state, p->d_partials);
  else
    k_direction_int<<<p->fx_blocks[kFxDir], p->st_block, 0, p->stream>>>(g, (const float*)p->d_Z, Pold, Pnew,
                                                                          p->d_state, p->d_partials);
}
void launch_update(const tpcg_plan* p, const Geom& g, double* U, int k, bool zero_guess_first) {
  LaunchScope ls(p, kKUpdate);
  if (p->prec == TPCG_FP64) {
    k_update<<<p->stream_blocks, 256, 0, p->stream>>>(g, U, (const double*)p->d_P[k & 1], p->d_W, p->d_R,
                                                       lowprec(p), p->d_state, p->d_partials);
    return;
  }
  const int slot = k % p->p_slots;
  const int* P = (const int*)p->d_P[slot];
  if (p->defer_u) {  // U += alpha P recorded for k_form_u
    if (g.nx % 2 == 0)
      k_update_pair<<<p->fx_blocks[kFxUpd], p->st_block, 0, p->stream>>>(g, P, p->d_R, lowprec(p), p->d_state,
                                                                          p->d_partials, slot);
    else
      k_update_int<<<p->fx_blocks[kFxUpd], p->st_block, 0, p->stream>>>(g, P, p->d_R, lowprec(p), p->d_state,
                                                                         p->d_partials, slot);
  } else if (g.nx % 2 == 0 && aligned16(U) && zero_guess_first) {  // first update of a zero guess: U = alpha P
    k_update_u_pair<true><<<p->fx_blocks[kFxUpd], p->st_block, 0, p->stream>>>(g, U, P, p->d_R, lowprec(p),
                                                                                p->d_state, p->d_partials);
  } else if (g.nx % 2 == 0 && aligned16(U)) {
    k_update_u_pair<false><<<p->fx_blocks[kFxUpd], p->st_block, 0, p->stream>>>(g, U, P, p->d_R, lowprec(p),
                                                                                 p->d_state, p->d_partials);
  } else if (zero_guess_first) {
    k_update_u_int<true><<<p->fx_blocks[kFxUpd], p->st_block, 0, p->stream>>>(g, U, P, p->d_R, lowprec(p),
                                                                               p->d_state, p->d_partials);
  } else {
    k_update_u_int<false><<<p->fx_blocks[kFxUpd], p->st_block, 0, p->stream>>>(g, U, P, p->d_R, lowprec(p),
                                                                                p->d_state, p->d_partials);
  }
}
// Mixed forms: apply the recorded updates to U (k_form_u) when a check is due, the ring is about to wrap,
// or (force) unconditionally.
void launch_form_u(const tpcg_plan* p, const Geom& g, double* U, bool force) {
  LaunchScope ls(p, kKFormU);
  if (g.N % 2 == 0 && aligned16(U))
    k_form_u<true><<<p->stream_blocks, 256, 0, p->stream>>>(g, U, (const int*)p->d_P[0], (unsigned long long)g.N,
                                                            p->d_state, p->d_partials, force ? 1 : 0);
  else
    k_form_u<false><<<p->stream_blocks, 256, 0, p->stream>>>(g, U, (const int*)p->d_P[0], (unsigned long long)g.N,
                                                             p->d_state, p->d_partials, force ? 1 : 0);
}
void launch_true_residual(const tpcg_plan* p, const Geom& g, const double* eta, const double* U, bool force) {
  LaunchScope ls(p, kKTrueRes);
  k_residual_fx<false><<<p->fx_blocks[kFxTrue], p->st_block, 0, p->stream>>>(g, eta, U, p->d_R, lowprec(p),
                                                                              p->d_state, p->d_partials, force ? 1 : 0);
}
void launch_center_u(const tpcg_plan* p, const Geom& g, double* U, int iter_lo) {
  LaunchScope ls(p, kKCenter);
  k_center_u<<<p->stream_blocks, 256, 0, p->stream>>>(g.N, U, p->d_state, iter_lo);
}
void launch_zero(const tpcg_plan* p, long long N, double* U) {
  LaunchScope ls(p, kKConvert);
  k_zero<<<p->stream_blocks, 256, 0, p->stream>>>(N, U);
}
void launch_to_lp(const tpcg_plan* p, const Geom& g, const double* r) {
  LaunchScope ls(p, kKConvert);
  k_to_lp<<<p->stream_blocks, 256, 0, p->stream>>>(g.N, r, lowprec(p), p->d_state);
}
void launch_f32_to_f64(const tpcg_plan* p, long long N, const float* a, double* b) {
  LaunchScope ls(p, kKConvert);
  k_f32_to_f64<<<p->stream_blocks, 256, 0, p->stream>>>(N, a, b);
}
void launch_fixed_to_f64(const tpcg_plan* p, long long N, const int* a, int kp, double* b) {
  LaunchScope ls(p, kKConvert);
  k_fixed_to_f64<<<p->stream_blocks, 256, 0, p->stream>>>(N, a, kp, b);
}
void launch_efield(const tpcg_plan* p, const Geom& g, const double* U, const double* bval, double* ex, double* ey,
                   double* ez) {
  LaunchScope ls(p, kKConvert);
  FaceData fd{};
  for (int m = 0; m < 6; ++m) fd.v[m] = bval ? bval[m] : 0.0;
  for (int m = 0; m < 3; ++m) {
    fd.h[m] = p->h[m];
    fd.inv2h[m] = 0.5 / p->h[m];
  }
  k_efield<<<p->stream_blocks, 256, 0, p->stream>>>(g, U, fd, ex, ey, ez);
}
// Comparator preconditioner of the FP64 form: Z = M(R), then (with st) rho, sum(Z) and the finalize.
void run_precond_cmp(const tpcg_plan* p, const Geom& g, const double* R, double* Z, SolveState* st) {
  if (p->pc_kind == TPCG_PRECOND_JACOBI) {
    JacobiTable t;
    for (int c = 0; c < 27; ++c) t.invd[c] = p->jac_invd[c];
    // X_j lands in Z when p - j is even, else in the W workspace, so that X_p is Z
    auto buf = [&](int j) { return ((p->jac_p - j) % 2 == 0) ? Z : p->d_W; };
    {
      LaunchScope ls(p, kKModeF64);
      k_jacobi_first<<<p->stream_blocks, 256, 0, p->stream>>>(g, R, buf(1), t);
    }
    for (int j = 2; j <= p->jac_p; ++j) {
      LaunchScope ls(p, kKModeF64);
      k_jacobi_sweep<<<p->st_grid, p->st_block, 0, p->stream>>>(g, p->st_zchunk, buf(j - 1), buf(j), R, t);
    }
  }
  if (st || p->pc_kind == TPCG_PRECOND_NONE) {
    LaunchScope ls(p, kKModeF64);
    k_dot_rz<<<p->stream_blocks, 256, 0, p->stream>>>(g.N, R, Z, p->pc_kind == TPCG_PRECOND_NONE ? 1 : 0, st,
                                                        p->d_partials);
  }
}

void launch_rhs_add_bc(const tpcg_plan* p, const Geom& g, double* eta, const double* bv) {
  LaunchScope ls(p, kKConvert);
  k_rhs_add_bc<<<p->stream_blocks, 256, 0, p->stream>>>(g, eta, bv[0], bv[1], bv[2], bv[3], bv[4], bv[5]);
}

}  // namespace tpcg
