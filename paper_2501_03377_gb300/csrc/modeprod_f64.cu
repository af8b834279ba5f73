// FP64 form of the pseudoinverse preconditioner (Algorithm 7, Sec. 4.3.3):
// six mode-product passes, each a GEMM that contracts the contiguous index of
// its input against a dense l x l eigenbasis matrix, with the Hadamard
// pseudoinverse G (Algorithm 5) recomputed in the epilogue of the
// last forward pass and the PCG reductions (<R, Z>, sum Z) fused into the
// epilogue of the last backward pass.
//
// FP64 has no tensor-core path on this part, so this is a register-blocked
// SIMT GEMM: 64 x 64 output tiles, 16-deep K slabs staged in shared memory,
// 4 x 4 outputs per thread.
#include "tpcg_dev.cuh"

namespace tpcg {

constexpr int MT = 64, NT = 64, KT = 16;

// Hadamard pseudoinverse entry G(a, b, c') = 1 / (lam_a + lam_b + lam_c'),
// zero at the (structural) null index (0, 0, 0) of a singular operator.
template <class T>
__device__ __forceinline__ T ghat(const T* la, const T* lb, const T* lc, int a, int b, int c, int singular) {
  if (singular && a == 0 && b == 0 && c == 0) return T(0);
  return T(1) / (la[a] + lb[b] + lc[c]);
}

struct ModeArgsF64 {
  StageParams p;
  const double* __restrict__ X;
  const double* __restrict__ Wm;   // C x Cout row-major
  double* __restrict__ Y;
  const double* lamA;
  const double* lamB;
  const double* lamC;
  int singular;
  // final stage only
  const double* __restrict__ R;
  SolveState* st;
  double* partials;
  long long N;
};

template <bool FINAL>
__global__ void __launch_bounds__(256) k_modeprod_f64(ModeArgsF64 a) {
  if (a.st && a.st->done) return;
  __shared__ double As[KT][MT + 2];
  __shared__ double Bs[KT][NT];
  const StageParams& p = a.p;
  const long long rows = (long long)p.A * p.B;
  const long long row0 = (long long)blockIdx.x * MT;
  const int col0 = blockIdx.y * NT;
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;

  for (int k0 = 0; k0 < p.C; k0 += KT) {
#pragma unroll
    for (int u = 0; u < (MT * KT) / 256; ++u) {
      const int e = tid + 256 * u;
      const int r = e / KT, kk = e % KT;
      const long long gr = row0 + r;
      const int gk = k0 + kk;
      As[kk][r] = (gr < rows && gk < p.C) ? __ldg(a.X + gr * p.in_pitch + gk) : 0.0;
    }
#pragma unroll
    for (int u = 0; u < (NT * KT) / 256; ++u) {
      const int e = tid + 256 * u;
      const int kk = e / NT, c = e % NT;
      const int gk = k0 + kk, gc = col0 + c;
      Bs[kk][c] = (gk < p.C && gc < p.Cout) ? __ldg(a.Wm + (long long)gk * p.Cout + gc) : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < KT; ++kk) {
      double av[4], bv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) av[i] = As[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bv[j] = Bs[kk][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
    }
    __syncthreads();
  }

  double red[2] = {0.0, 0.0};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const long long gr = row0 + ty * 4 + i;
    if (gr >= rows) continue;
    const int aa = (int)(gr / p.B), bb = (int)(gr - (long long)aa * p.B);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gc = col0 + tx * 4 + j;
      if (gc >= p.Cout) continue;
      double v = acc[i][j];
      if (p.scale) v *= ghat<double>(a.lamA, a.lamB, a.lamC, aa, bb, gc, a.singular);
      const long long o = (long long)aa * p.oa + (long long)bb * p.ob + (long long)gc * p.oc;
      a.Y[o] = v;
      if (FINAL) {
        red[0] = fma(__ldg(a.R + o), v, red[0]);
        red[1] += v;
      }
    }
  }
  if constexpr (FINAL) {
    SolveState* st = a.st;
    const long long N = a.N;
    grid_reduce<2>(red, a.partials, &st->tickets[kTkPrec], gridDim.x * gridDim.y, blockIdx.x + gridDim.x * blockIdx.y,
                   [st, N](const double(&s)[2]) { fin_precond(st, N, s); });
  }
}

// Runs the whole FP64 preconditioner: R (FP64, unpadded) -> Z (FP64).  With
// st != nullptr the last pass also performs the PCG finalize.
void run_precond_f64(const tpcg_plan* pl, const double* R, double* Z, SolveState* st) {
  const int ns = (int)pl->stages.size();
  const double* in = R;
  for (int s = 0; s < ns; ++s) {
    const StageParams& p = pl->stages[s];
    ModeArgsF64 a{};
    a.p = p;
    a.X = in;
    a.Wm = pl->d_W64[p.axis][p.dir];
    const bool last = (s == ns - 1);
    a.Y = last ? Z : (double*)pl->d_T[s & 1];
    a.lamA = pl->d_lam64[p.lamA];
    a.lamB = pl->d_lam64[p.lamB];
    a.lamC = pl->d_lam64[p.lamC];
    a.singular = pl->singular ? 1 : 0;
    a.R = R;
    a.st = st;
    a.partials = pl->d_partials;
    a.N = pl->N;
    const long long rows = (long long)p.A * p.B;
    dim3 grid((unsigned)((rows + MT - 1) / MT), (unsigned)((p.Cout + NT - 1) / NT));
    LaunchScope ls(pl, kKModeF64);
    if (last && st)
      k_modeprod_f64<true><<<grid, 256, 0, pl->stream>>>(a);
    else
      k_modeprod_f64<false><<<grid, 256, 0, pl->stream>>>(a);
    in = a.Y;
  }
}

}  // namespace tpcg
