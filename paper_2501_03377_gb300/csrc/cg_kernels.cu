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

template <class ZT>
struct FieldDirection {  // P = (Z - mean Z) + beta * P_old   (Algorithm 1, line 17; Remark orthogonality)
  const ZT* __restrict__ z;
  const double* __restrict__ pold;
  double mZ, beta;
  int first;
  __device__ __forceinline__ double operator()(long long i) const {
    double zi;
    if constexpr (sizeof(ZT) == 4)
      zi = f32_to_f64_int(__ldg(reinterpret_cast<const float*>(z) + i));
    else
      zi = __ldg(reinterpret_cast<const double*>(z) + i);
    zi -= mZ;
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
// Input of the first tensor-core pass: BF16, or FP16 of R * 2^shift, rows
// padded to `pitch` elements.  ptr == nullptr in the FP64 form.
struct LowPrec {
  void* ptr;
  int kind;  // 1 BF16, 2 FP16
  int pitch, nx;
};

__device__ __forceinline__ void store_lp(const LowPrec& lp, int shift, long long i, double r) {
  if (!lp.ptr) return;
  long long j = i;
  if (lp.pitch != lp.nx) {
    const long long row = i / lp.nx;
    j = row * lp.pitch + (i - row * lp.nx);
  }
  reinterpret_cast<uint16_t*>(lp.ptr)[j] = (lp.kind == 2) ? f64_to_f16_bits(r, shift) : f64_to_bf16_bits(r);
}

// ------------------------------------------------------------------ residual R = eta_hat - L U
// Used for the initial residual (Algorithm 1, lines 3-4) and the FP64 check of
// the true residual (stop test); the latter replaces R (residual replacement)
// and accumulates sum(U) for the exit centring.
struct OpResidual {
  const double* __restrict__ eta;
  double* __restrict__ R;
  LowPrec lp;
  int shift;
  double mean;
  __device__ __forceinline__ void operator()(long long i, double c, double w, double (&acc)[4]) {
    const double e = __ldg(eta + i) - mean;
    const double r = e - w;
    R[i] = r;
    store_lp(lp, shift, i, r);
    acc[0] = fma(r, r, acc[0]);
    acc[1] += r;
    acc[2] = fma(e, e, acc[2]);
    acc[3] += c;
  }
};

// The low-precision copy just written used lp_shift; the next one uses the
// exponent that scales the new residual to unit RMS.
__device__ __forceinline__ void advance_shift(SolveState* st, double rr, long long N) {
  st->lp_shift_applied = st->lp_shift;
  st->lp_shift = lp_shift_for(rr, N);
}

__device__ void fin_init(SolveState* st, const double (&s)[4], long long N) {
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

__global__ void __launch_bounds__(TX* TY) k_init_residual(Geom g, int zchunk, const double* __restrict__ eta,
                                                          const double* __restrict__ U, double* __restrict__ R,
                                                          LowPrec lp, SolveState* st, double* partials) {
  FieldPlain f{U};
  OpResidual op{eta, R, lp, st->lp_shift, st->mean_eta};
  const long long N = g.N;
  stencil_sweep<4>(g, zchunk, f, op, partials, &st->tickets[kTkInit],
                   [st, N](const double(&s)[4]) { fin_init(st, s, N); });
}

__device__ void fin_true(SolveState* st, const double (&s)[4], long long N) {
  st->true_rr = s[0];
  st->sumU = s[3];
  advance_shift(st, s[0], N);
  if (!isfinite(s[0])) {
    st->status = TPCG_ERR_BREAKDOWN;
    st->done = 1;
    return;
  }
  if (s[0] <= st->tol2) {
    st->status = TPCG_OK;
    st->done = 1;
  } else if (st->iter >= st->maxit) {
    st->status = TPCG_ERR_NOT_CONVERGED;
    st->done = 1;
  } else {  // keep iterating from the replaced (true) residual
    st->rr = s[0];
    st->sumR = s[1];
    st->need_check = 0;
  }
}

__global__ void __launch_bounds__(TX* TY) k_true_residual(Geom g, int zchunk, const double* __restrict__ eta,
                                                          const double* __restrict__ U, double* __restrict__ R,
                                                          LowPrec lp, SolveState* st, double* partials, int force) {
  if (!force && (st->done || !st->need_check)) return;
  FieldPlain f{U};
  OpResidual op{eta, R, lp, st->lp_shift, st->mean_eta};
  const long long N = g.N;
  stencil_sweep<4>(g, zchunk, f, op, partials, &st->tickets[kTkTrue],
                   [st, force, N](const double(&s)[4]) {
                     if (force) {
                       st->true_rr = s[0];
                       st->sumU = s[3];
                     } else {
                       fin_true(st, s, N);
                     }
                   });
}

// ------------------------------------------------------------------ direction + W = L P
// P_s = Z_s' + beta_s P_{s-1} (line 17, with Z centred), W = L P (line 10),
// <W, P> and alpha = rho / <W, P> (line 11).
struct OpDirection {
  double* __restrict__ P;
  double* __restrict__ W;
  __device__ __forceinline__ void operator()(long long i, double c, double w, double (&acc)[1]) {
    P[i] = c;
    W[i] = w;
    acc[0] = fma(w, c, acc[0]);
  }
};

__device__ void fin_direction(SolveState* st, const double (&s)[1]) {
  st->pWp = s[0];
  st->first = 0;
  if (!(s[0] > 0.0) || !isfinite(s[0])) {
    st->status = TPCG_ERR_BREAKDOWN;
    st->done = 1;
    return;
  }
  st->alpha = st->rho / s[0];
}

template <class ZT>
__global__ void __launch_bounds__(TX* TY) k_direction(Geom g, int zchunk, const ZT* __restrict__ Z,
                                                      const double* __restrict__ Pold, double* __restrict__ P,
                                                      double* __restrict__ W, SolveState* st, double* partials) {
  if (st->done) return;
  FieldDirection<ZT> f{Z, Pold, st->mZ, st->beta, st->first};
  OpDirection op{P, W};
  stencil_sweep<1>(g, zchunk, f, op, partials, &st->tickets[kTkDir],
                   [st](const double(&s)[1]) { fin_direction(st, s); });
}

// ------------------------------------------------------------------ direction, mixed forms
// Z arrives in FP32.  It enters the stencil as exact fixed point
// round(Z * 2^k) (int32, |.| < 2^27, k from max|Z| of the preconditioner
// output), so the second differences are exact integers and
//     W_s = L P_s = L Z_s + beta_s W_{s-1}        (Algorithm 1, lines 10, 17)
// needs only two FP64 FMAs per point besides <W, P>.  P_s = Z_s + beta P_{s-1}
// keeps the constant (null-space) component of Z: L annihilates it, so W and
// <W, P> are those of the centred Z (Remark orthogonality), rho is corrected by
// -mean(Z) sum(R), and the resulting constant offset of U is removed at exit.
template <int NQ, class Field, class Op, class Fin>
__device__ __forceinline__ void stencil_sweep_int(const Geom& g, int zchunk, const Field& field, Op& op,
                                                  double* partials, unsigned* ticket, Fin fin) {
  __shared__ int ring[4][SY][SX];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * TX + tx;
  const int bx0 = blockIdx.x * TX, by0 = blockIdx.y * TY;
  const int x = bx0 + tx, y = by0 + ty;
  const int k0 = blockIdx.z * zchunk;
  const int k1 = min(g.nz, k0 + zchunk);
  const bool active = (x < g.nx) && (y < g.ny);
  const bool has_z = g.nz > 1;
  const long long plane = (long long)g.nx * g.ny;
  double acc[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) acc[q] = 0.0;

  auto load_plane = [&](int kk) {
    const int kz = has_z ? ghost_index(kk, g.nz, g.bc[2]) : kk;
    int(*dst)[SX] = ring[kk & 3];
    for (int e = tid; e < SX * SY; e += TX * TY) {
      const int sx = e % SX, sy = e / SX;
      const int gx = ghost_index(bx0 + sx - 1, g.nx, g.bc[0]);
      const int gy = ghost_index(by0 + sy - 1, g.ny, g.bc[1]);
      int v = 0;
      if (kz >= 0 && gx >= 0 && gy >= 0) v = field((long long)kz * plane + (long long)gy * g.nx + gx);
      dst[sy][sx] = v;
    }
  };

  if (k0 < k1) {
    if (has_z) load_plane(k0 - 1);
    load_plane(k0);
    for (int k = k0; k < k1; ++k) {
      if (has_z) load_plane(k + 1);
      __syncthreads();
      if (active) {
        const int(*cur)[SX] = ring[k & 3];
        const int c = cur[ty + 1][tx + 1];
        const int dx = 2 * c - cur[ty + 1][tx] - cur[ty + 1][tx + 2];
        const int dy = 2 * c - cur[ty][tx + 1] - cur[ty + 2][tx + 1];
        const int dz = has_z ? 2 * c - ring[(k - 1) & 3][ty + 1][tx + 1] - ring[(k + 1) & 3][ty + 1][tx + 1] : 0;
        op((long long)k * plane + (long long)y * g.nx + x, c, dx, dy, dz, acc);
      }
    }
  }
  const int nblocks = gridDim.x * gridDim.y * gridDim.z;
  const int bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
  grid_reduce<NQ>(acc, partials, ticket, nblocks, bid, fin);
}

struct FieldFixed {
  const float* __restrict__ z;
  int k;
  __device__ __forceinline__ int operator()(long long i) const { return f32_to_fixed(__ldg(z + i), k); }
};

struct OpDirectionFx {
  const double* pold;
  const double* wold;
  double* p;
  double* w;
  double beta, ih0, ih1, ih2;
  int first, e, uniform;
  __device__ __forceinline__ void operator()(long long i, int c, int dx, int dy, int dz, double (&acc)[1]) {
    const double zf = i32_to_f64_scaled(c, e);
    double lz;
    if (uniform) {
      lz = i32_to_f64_scaled(dx + dy + dz, e);
      if (ih0 != 1.0) lz *= ih0;
    } else {
      lz = fma(i32_to_f64_scaled(dx, e), ih0, i32_to_f64_scaled(dy, e) * ih1);
      if (dz) lz = fma(i32_to_f64_scaled(dz, e), ih2, lz);
    }
    const double pv = first ? zf : fma(beta, __ldg(pold + i), zf);
    const double wv = first ? lz : fma(beta, wold[i], lz);
    p[i] = pv;
    w[i] = wv;
    acc[0] = fma(wv, pv, acc[0]);
  }
};

__global__ void __launch_bounds__(TX* TY) k_direction_fx(Geom g, int zchunk, const float* __restrict__ Z,
                                                         const double* Pold, double* P, double* W, SolveState* st,
                                                         double* partials) {
  if (st->done) return;
  const int k = st->zfx_shift;
  FieldFixed f{Z, k};
  const bool has_z = g.nz > 1;
  const int uniform = (g.ih2[0] == g.ih2[1]) && (!has_z || g.ih2[2] == g.ih2[0]);
  OpDirectionFx op{Pold, W, P, W, st->beta, g.ih2[0], g.ih2[1], g.ih2[2], st->first, -k, uniform};
  stencil_sweep_int<1>(g, zchunk, f, op, partials, &st->tickets[kTkDir],
                       [st](const double(&s)[1]) { fin_direction(st, s); });
}

// ------------------------------------------------------------------ streaming kernels
// U += alpha P (line 12), R -= alpha W (line 13), low-precision copy of R,
// ||R||^2 and sum(R) for the stop test and the centring correction of rho.
// The two sums are accumulated per thread in FP32 from R * 2^lp_shift (exact
// power-of-two scaling, unit RMS) and combined across threads in FP64: they
// only steer the stop test, which the FP64 true residual confirms.
__device__ void fin_update(SolveState* st, const double (&s)[2], int shift, long long N) {
  const double rr = ldexp(s[0], -2 * shift), sumR = ldexp(s[1], -shift);
  st->rr = rr;
  st->sumR = sumR;
  st->iter += 1;
  st->zero_guess = 0;
  advance_shift(st, rr, N);
  if (!isfinite(rr)) {
    st->status = TPCG_ERR_BREAKDOWN;
    st->done = 1;
    return;
  }
  if (rr <= st->tol2 || st->iter >= st->maxit) st->need_check = 1;
}

__global__ void __launch_bounds__(256) k_update(long long N, double* __restrict__ U, const double* __restrict__ P,
                                                const double* __restrict__ W, double* __restrict__ R, LowPrec lp,
                                                SolveState* st, double* partials) {
  if (st->done) return;
  const double alpha = st->alpha;
  const double nalpha = -alpha;
  const int zg = st->zero_guess;
  const int shift = st->lp_shift;
  float a0 = 0.0f, a1 = 0.0f;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    const double p = __ldg(P + i);
    U[i] = zg ? alpha * p : fma(alpha, p, U[i]);
    const double r = fma(nalpha, __ldg(W + i), R[i]);
    R[i] = r;
    store_lp(lp, shift, i, r);
    const float r32 = f64_to_f32_int(r, shift);
    a0 = fmaf(r32, r32, a0);
    a1 += r32;
  }
  double acc[2] = {(double)a0, (double)a1};
  grid_reduce<2>(acc, partials, &st->tickets[kTkUpd], gridDim.x, blockIdx.x,
                 [st, shift, N](const double(&s)[2]) { fin_update(st, s, shift, N); });
}

// R = eta_hat (zero initial guess: lines 3-4 with U_0 = 0).
__global__ void __launch_bounds__(256) k_init_zero(long long N, const double* __restrict__ eta,
                                                   double* __restrict__ R, LowPrec lp, SolveState* st,
                                                   double* partials) {
  const double mean = st->mean_eta;
  const int shift = st->lp_shift;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    const double r = __ldg(eta + i) - mean;
    R[i] = r;
    store_lp(lp, shift, i, r);
    acc[0] = fma(r, r, acc[0]);
    acc[1] += r;
  }
  acc[2] = acc[0];
  grid_reduce<4>(acc, partials, &st->tickets[kTkInit], gridDim.x, blockIdx.x,
                 [st, N](const double(&s)[4]) { fin_init(st, s, N); });
}

// sum(eta) and sum(eta^2): the mean removed by eq. (centering) when the
// operator is singular, and the exponent of the first low-precision copy.
__global__ void __launch_bounds__(256) k_eta_sum(long long N, const double* __restrict__ eta, SolveState* st,
                                                 double* partials) {
  double acc[2] = {0.0, 0.0};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    const double e = __ldg(eta + i);
    acc[0] += e;
    acc[1] = fma(e, e, acc[1]);
  }
  grid_reduce<2>(acc, partials, &st->tickets[kTkEta], gridDim.x, blockIdx.x, [st, N](const double(&s)[2]) {
    const double mean = st->singular ? s[0] / (double)N : 0.0;
    st->mean_eta = mean;
    const double n2 = s[1] - mean * s[0];
    st->lp_shift = lp_shift_for(n2 > 0.0 ? n2 : s[1], N);
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

// U -= sum(U)/N: return the zero-mean (minimum-norm) representative.
__global__ void __launch_bounds__(256) k_center_u(long long N, double* __restrict__ U, const SolveState* st) {
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
    store_lp(lp, shift, i, __ldg(r + i));
  if (blockIdx.x == 0 && threadIdx.x == 0) st->lp_shift_applied = shift;
}

// FP32 -> FP64 copy (Z of the mixed forms, for tpcg_precond_apply).
__global__ void __launch_bounds__(256) k_f32_to_f64(long long N, const float* __restrict__ a, double* __restrict__ b) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x)
    b[i] = f32_to_f64_int(__ldg(a + i));
}

// Sec. 3.4.2: fold constant boundary data into the right-hand side.  bval[2m]
// at the start face of axis m, bval[2m+1] at the end face; Dirichlet adds
// u/h^2 to the boundary layer, Neumann adds e/h (e: outward derivative).
__global__ void k_rhs_add_bc(Geom g, double* __restrict__ eta, double b0, double b1, double b2, double b3, double b4,
                             double b5) {
  const double bv[6] = {b0, b1, b2, b3, b4, b5};
  const long long plane = (long long)g.nx * g.ny;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < g.N; i += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(i / plane);
    const long long rem = i - (long long)k * plane;
    const int y = (int)(rem / g.nx), x = (int)(rem - (long long)y * g.nx);
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

// ------------------------------------------------------------------ host launchers
void launch_apply_laplacian(const tpcg_plan* p, const Geom& g, const double* x, double* w) {
  LaunchScope ls(p, kKApply);
  k_apply_laplacian<<<p->st_grid, p->st_block, 0, p->stream>>>(g, p->st_zchunk, x, w);
}
LowPrec lowprec(const tpcg_plan* p) { return LowPrec{p->d_Rlp, p->lp_kind, p->pitch16[0], p->nx}; }

void launch_init_residual(const tpcg_plan* p, const Geom& g, const double* eta, const double* U, bool zero_guess) {
  LaunchScope ls(p, kKInit);
  if (zero_guess)
    k_init_zero<<<p->stream_blocks, 256, 0, p->stream>>>(g.N, eta, p->d_R, lowprec(p), p->d_state, p->d_partials);
  else
    k_init_residual<<<p->st_grid, p->st_block, 0, p->stream>>>(g, p->st_zchunk, eta, U, p->d_R, lowprec(p),
                                                                p->d_state, p->d_partials);
}
void launch_eta_sum(const tpcg_plan* p, const Geom& g, const double* eta) {
  LaunchScope ls(p, kKEtaSum);
  k_eta_sum<<<p->stream_blocks, 256, 0, p->stream>>>(g.N, eta, p->d_state, p->d_partials);
}
void launch_norm_shift(const tpcg_plan* p, const Geom& g, const double* r) {
  LaunchScope ls(p, kKConvert);
  k_norm_shift<<<p->stream_blocks, 256, 0, p->stream>>>(g.N, r, p->d_state, p->d_partials);
}
void launch_direction(const tpcg_plan* p, const Geom& g, int k) {
  LaunchScope ls(p, kKDirection);
  const double* pold = p->d_P[(k + 1) & 1];
  double* pnew = p->d_P[k & 1];
  if (p->prec == TPCG_FP64)
    k_direction<double><<<p->st_grid, p->st_block, 0, p->stream>>>(g, p->st_zchunk, (const double*)p->d_Z, pold, pnew,
                                                                    p->d_W, p->d_state, p->d_partials);
  else
    k_direction_fx<<<p->st_grid, p->st_block, 0, p->stream>>>(g, p->st_zchunk, (const float*)p->d_Z, pold, pnew,
                                                               p->d_W, p->d_state, p->d_partials);
}
void launch_update(const tpcg_plan* p, const Geom& g, double* U, int k) {
  LaunchScope ls(p, kKUpdate);
  k_update<<<p->stream_blocks, 256, 0, p->stream>>>(g.N, U, p->d_P[k & 1], p->d_W, p->d_R, lowprec(p), p->d_state,
                                                     p->d_partials);
}
void launch_true_residual(const tpcg_plan* p, const Geom& g, const double* eta, const double* U, bool force) {
  LaunchScope ls(p, kKTrueRes);
  k_true_residual<<<p->st_grid, p->st_block, 0, p->stream>>>(g, p->st_zchunk, eta, U, p->d_R, lowprec(p), p->d_state,
                                                              p->d_partials, force ? 1 : 0);
}
void launch_center_u(const tpcg_plan* p, const Geom& g, double* U) {
  LaunchScope ls(p, kKCenter);
  k_center_u<<<p->stream_blocks, 256, 0, p->stream>>>(g.N, U, p->d_state);
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
void launch_rhs_add_bc(const tpcg_plan* p, const Geom& g, double* eta, const double* bv) {
  LaunchScope ls(p, kKConvert);
  k_rhs_add_bc<<<p->stream_blocks, 256, 0, p->stream>>>(g, eta, bv[0], bv[1], bv[2], bv[3], bv[4], bv[5]);
}

}  // namespace tpcg
