// Mixed-precision forms of the pseudoinverse preconditioner (Algorithm 7,
// Sec. 4.3.3) on the 5th-generation tensor cores: every mode-product pass is
// a tcgen05 GEMM (FP16, BF16, TF32, or split BF16 pairs; FP32 accumulation)
// that contracts the contiguous index of its input against the l x l
// eigenbasis.
//
// One persistent, warp-specialised kernel serves every single pass:
//   warp 0      TMA producer: loads the eigenbasis W^T (K-major, 128B-
//               swizzled) into shared memory once, then streams 128-row x
//               128-byte K-tiles of the input through an NS-slot ring (the
//               4-byte forms -- TF32 and the split BF16 pairs -- stream the
//               eigenbasis K-tile with each data K-tile instead);
//   warp 1      allocates TMEM; lane 0 issues tcgen05.mma (M = 128) and
//               tcgen05.commit to release ring slots / publish accumulators;
//   warps 2..9  epilogue: tcgen05.ld of the FP32 accumulator (one TMEM lane
//               per thread), optional Hadamard scaling by G = 1/(lam_a +
//               lam_b + lam_c) with the null index zeroed (Algorithm 5),
//               FP16/BF16 (or FP32) stores, and in the last pass the PCG
//               reductions <R, Z>, sum Z and max |Z|.
// Two accumulator buffers in TMEM let the epilogue of tile i overlap the MMAs
// of tile i+1.  Two operand forms keep the global stores coalesced:
//   form 1: D[row][c'] = X[row][:] . W^T[c'][:]  (data = A, M = 128 rows,
//           eigenbasis = B, N = Cout padded to 16); lanes walk the rows;
//   form 2: D[c'][row] = W^T[c'][:] . X[row][:]  (eigenbasis = A in M-blocks
//           of 128, data = B, N = 128); lanes walk the output index.
// A second kernel, k_modeprod_pair, runs the forward and the backward pass
// along the axis of the Hadamard step as one launch (see its comment); the
// plan uses it where the layout allows and the option TPCG_OPT_FUSE_G is on.
// Every wait on an mbarrier is bounded (globaltimer); on expiry the CTA sets
// an error word, stops issuing, drains its own copies/MMAs with bounded waits,
// frees TMEM and returns.
#include <cuda.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>
#include <type_traits>
#include <cstdio>
#include <vector>

#include "tc_ptx.cuh"

namespace tpcg {

namespace {
using namespace tcx;

// Warp roles: warp 0 TMA of the operand, warp 1 MMA, then the epilogue warps, one group of four per
// share of the accumulator's 16-column chunks (a warp may only read its TMEM lane quadrant, warp % 4).
// The plain passes use sixteen epilogue warps; the last pass of a solve keeps eight, plus one warp
// that stages R by TMA.
template <bool FINAL>
struct TcWarps {
  static constexpr int epi = FINAL ? 8 : 16;
  static constexpr int groups = epi / 4;
  static constexpr int threads = (2 + epi + (FINAL ? 1 : 0)) * 32;
  static constexpr int rwarp = FINAL ? 2 + epi : -1;
};
constexpr int kRSlots = 16;                // R chunks in flight (last pass): eight slots per epilogue half
constexpr int kRHalf = kRSlots / 2;
constexpr int kRBytes = 128 * 16 * 2;      // one chunk: 128 rows x 16 FP16/BF16 columns
constexpr int kTileRows = 128;
constexpr int kKTile = 64;                 // BF16 elements per 128-byte swizzle row
constexpr int kStageBytes = kTileRows * 128;

// The split form's operand type: x carried as two BF16 planes, hi = bf16(x) and lo = bf16(x - hi).  A stage
// holds the hi tile and then the lo tile of the data (and of the eigenbasis), and every K step issues three
// MMAs into one FP32 accumulator: hi.hi + lo.hi + hi.lo (the lo.lo term, 2^-16 relative, is dropped).
struct Bf16Pair {};

// Elements of InT per 128-byte swizzle row (one K tile) and per MMA K step.
template <class InT>
struct KShape {
  static constexpr bool tf32 = sizeof(InT) == 4;
  static constexpr bool split = false;
  static constexpr int tile = 128 / (int)sizeof(InT);  // 64 (FP16/BF16) or 32 (TF32)
  static constexpr int step = tf32 ? 8 : 16;
};
template <>
struct KShape<Bf16Pair> {
  static constexpr bool tf32 = false;
  static constexpr bool split = true;
  static constexpr int tile = 64;
  static constexpr int step = 16;
};

struct TcArgs {
  int C, KT, Cout, VR, Np, MB, acc_cols, tmem_cols, NS;
  int rows, B;
  int B1;  // fused pair: the row split (a, b) of the forward pass, for G
  long long oa, ob, oc;
  int scale, singular;
  int vec;   // 16-element runs of the output are contiguous and 16-byte aligned
  int rtma;  // last pass: R~ arrives by TMA, else by global loads
  int rhalf;   // R~ ring slots per epilogue half (last pass, rtma)
  int tstore;  // outputs leave through shared memory by TMA stores (tmO), else by direct stores
  int tperm;   // form 2 output map: dims {B, A, Cout} (1) or {B, Cout, A} (0)
  int aux;     // bytes of shared memory after the stages: R~ ring (last pass) and output staging
  int wstream;  // eigenbasis K tiles streamed with the data tiles (each stage holds both), else resident
  int sbytes;   // bytes of one stage (data tile, plus the eigenbasis tile when streamed; split: hi and lo of each)
  int last;  // last pass: output is Z (FP32), undo the FP16 scaling
  int sG;    // the Hadamard step is multiplied by 2^-sG (FP16 range), undone on Z
  float gscale;          // 2^-sG
  const int* shift_src;  // exponent the FP16 copy of R was scaled with (device)
  const float* lamA;
  const float* lamB;
  const float* lamC;
  void* out;
  const uint16_t* Rt;  // the tensor-core copy of R the first pass read (FP16 = R * 2^shR, BF16 = R, TF32 = R
                       // in FP32 containers, or the hi plane of the split pair of R * 2^shR)
  int rpitch;          // its row pitch (elements)
  long long rplane;    // split form: 16-bit words from the hi plane of R~ to its lo plane
  long long oplane;    // split form: 16-bit words from the hi plane of the output to its lo plane
  SolveState* st;
  double* partials;
  long long N;
  int* err;
};

// 32 bytes to a 32-byte aligned global address in one store (a whole sector).
__device__ __forceinline__ void st_global_v8(void* p, const uint32_t (&w)[8]) {
  asm volatile("st.global.v8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p), "r"(w[0]), "r"(w[1]), "r"(w[2]),
               "r"(w[3]), "r"(w[4]), "r"(w[5]), "r"(w[6]), "r"(w[7])
               : "memory");
}

// hi = bf16(v) at o, lo = bf16(v - hi) one plane further (v - hi is exact in FP32).
__device__ __forceinline__ void store_pair(void* out, long long plane, long long o, float v) {
  const __nv_bfloat16 hi = __float2bfloat16_rn(v);
  reinterpret_cast<__nv_bfloat16*>(out)[o] = hi;
  reinterpret_cast<__nv_bfloat16*>(out)[plane + o] = __float2bfloat16_rn(v - __bfloat162float(hi));
}

template <class OutT>
__device__ __forceinline__ void store_out(void* out, long long plane, long long o, float v) {
  if constexpr (std::is_same<OutT, Bf16Pair>::value)
    store_pair(out, plane, o, v);
  else if constexpr (std::is_same<OutT, __half>::value)
    reinterpret_cast<__half*>(out)[o] = __float2half_rn(v);
  else if constexpr (sizeof(OutT) == 2)
    reinterpret_cast<__nv_bfloat16*>(out)[o] = __float2bfloat16_rn(v);
  else
    reinterpret_cast<float*>(out)[o] = v;
}

// 16 consecutive outputs starting at element offset o (16-byte aligned); the split form writes the hi
// words at o and the lo words one plane further.
template <class OutT>
__device__ __forceinline__ void store16(void* out, long long plane, long long o, const float (&x)[16]) {
  if constexpr (std::is_same<OutT, Bf16Pair>::value) {
    uint32_t ph[8], pl[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const __nv_bfloat162 h2 = __floats2bfloat162_rn(x[2 * i], x[2 * i + 1]);
      const float2 hf = __bfloat1622float2(h2);
      const __nv_bfloat162 l2 = __floats2bfloat162_rn(x[2 * i] - hf.x, x[2 * i + 1] - hf.y);
      ph[i] = *reinterpret_cast<const uint32_t*>(&h2);
      pl[i] = *reinterpret_cast<const uint32_t*>(&l2);
    }
    uint16_t* dh = reinterpret_cast<uint16_t*>(out) + o;
    uint16_t* dl = reinterpret_cast<uint16_t*>(out) + plane + o;
    if ((o & 15) == 0 && (plane & 15) == 0) {  // 32-byte aligned: one full sector per store
      st_global_v8(dh, ph);
      st_global_v8(dl, pl);
    } else {
      reinterpret_cast<uint4*>(dh)[0] = make_uint4(ph[0], ph[1], ph[2], ph[3]);
      reinterpret_cast<uint4*>(dh)[1] = make_uint4(ph[4], ph[5], ph[6], ph[7]);
      reinterpret_cast<uint4*>(dl)[0] = make_uint4(pl[0], pl[1], pl[2], pl[3]);
      reinterpret_cast<uint4*>(dl)[1] = make_uint4(pl[4], pl[5], pl[6], pl[7]);
    }
  } else if constexpr (sizeof(OutT) == 2) {
    uint32_t pk[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      if constexpr (std::is_same<OutT, __half>::value) {
        __half2 h2 = __floats2half2_rn(x[2 * i], x[2 * i + 1]);
        pk[i] = *reinterpret_cast<uint32_t*>(&h2);
      } else {
        __nv_bfloat162 h2 = __floats2bfloat162_rn(x[2 * i], x[2 * i + 1]);
        pk[i] = *reinterpret_cast<uint32_t*>(&h2);
      }
    }
    uint4* d = reinterpret_cast<uint4*>(reinterpret_cast<uint16_t*>(out) + o);
    d[0] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
    d[1] = make_uint4(pk[4], pk[5], pk[6], pk[7]);
  } else {
    float4* d = reinterpret_cast<float4*>(reinterpret_cast<float*>(out) + o);
#pragma unroll
    for (int i = 0; i < 4; ++i) d[i] = make_float4(x[4 * i], x[4 * i + 1], x[4 * i + 2], x[4 * i + 3]);
  }
}

template <int FORM, class InT, class OutT, bool FINAL>
__global__ void __launch_bounds__(TcWarps<FINAL>::threads, 1)
    k_modeprod_tc(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmW,
                  const __grid_constant__ CUtensorMap tmR, const __grid_constant__ CUtensorMap tmO, TcArgs a) {
  if (a.st && a.st->done) return;
  // Programmatic dependent launch: the next pass may start its prologue (barriers, TMEM, eigenbasis
  // load) on SMs this grid frees; it waits (griddepcontrol.wait) before touching this pass's output.
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t* sm = smem_raw + (base - raw);
  using KS = KShape<InT>;
  const uint32_t sV = base;
  const uint32_t vres = a.wstream ? 0u : (uint32_t)a.KT * a.VR * 128u;  // resident eigenbasis
  const uint32_t sD = sV + vres;
  const uint32_t sbytes = (uint32_t)a.sbytes;
  const bool rtma = FINAL && a.rtma;
  const uint32_t sR = sD + (uint32_t)a.NS * sbytes;  // 1024-aligned: V and stages are multiples of 1 KB
  // output staging: two [32][16] boxes per epilogue warp, after the R~ ring of the last pass (the split
  // form stores directly)
  using StageT = typename std::conditional<std::is_same<OutT, Bf16Pair>::value, __nv_bfloat16, OutT>::type;
  constexpr uint32_t kOBytes = 32u * 16u * (uint32_t)sizeof(StageT);
  const uint32_t sO = sR + (rtma ? (uint32_t)(2 * a.rhalf * kRBytes) : 0u);
  uint8_t* barp = sm + (size_t)vres + (size_t)a.NS * sbytes + (size_t)a.aux;
  const uint32_t bars = smem_u32(barp);
  const int NS = a.NS;
  auto full = [&](int s) { return bars + 8u * s; };
  auto empty = [&](int s) { return bars + 8u * (NS + s); };
  auto tfull = [&](int b) { return bars + 8u * (2 * NS + b); };
  auto tempty = [&](int b) { return bars + 8u * (2 * NS + 2 + b); };
  const uint32_t vbar = bars + 8u * (2 * NS + 4);
  const uint32_t drain = bars + 8u * (2 * NS + 5);
  auto rfull = [&](int s) { return bars + 8u * (2 * NS + 6 + s); };
  auto rempty = [&](int s) { return bars + 8u * (2 * NS + 6 + kRSlots + s); };
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(barp + 8 * (2 * NS + 6 + 2 * kRSlots));
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_holder + 1);
  const Abort ab{abort_flag, a.err, a.st};

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < NS; ++s) {
      mbar_init(full(s), 1);
      mbar_init(empty(s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(tfull(b), 1);
      mbar_init(tempty(b), TcWarps<FINAL>::epi * 32);
    }
    mbar_init(vbar, 1);
    mbar_init(drain, 1);
    for (int s = 0; s < kRSlots; ++s) {
      mbar_init(rfull(s), 1);
      mbar_init(rempty(s), TcWarps<FINAL>::epi * 16);  // the warps of one epilogue half
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_holder)),
                 "r"((uint32_t)a.tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_holder;
  const int ntiles = (a.rows + kTileRows - 1) / kTileRows;

  // last pass: rho = <R~, Z>, R~ the copy of R the first pass consumed (FP16 and split: R * 2^shR; BF16 and
  // TF32: R, brought to the same 2^shR scale), from FP32 products in compensated FP32 per thread; sum(Z)
  // likewise; max |Z|
  Acc32 red0, red1;
  float zmax = 0.0f;
  const int shR = (FINAL && a.st) ? a.st->lp_shift_applied : 0;
  const float rs = (std::is_same<InT, __half>::value || KS::split) ? 1.0f : ldexpf(1.0f, shR);
  const uint16_t* Rlo = KS::split ? a.Rt + a.rplane : nullptr;  // split form: lo plane of R~

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer
      if (!a.wstream) {
        mbar_expect_tx(vbar, vres);
        for (int kt = 0; kt < a.KT; ++kt) tma_load_2d(sV + (uint32_t)kt * a.VR * 128u, &tmW, kt * KS::tile, 0, vbar);
      }
      // the operand is the previous pass's output: wait until that grid has completed
      asm volatile("griddepcontrol.wait;" ::: "memory");
      int it = 0;
      for (int tile = blockIdx.x; tile < ntiles && !*abort_flag; tile += gridDim.x) {
        for (int kt = 0; kt < a.KT; ++kt, ++it) {
          const int s = it % NS;
          const uint32_t ph = (uint32_t)((it / NS) & 1);
          if (!wait_bounded(empty(s), ph ^ 1u, ab)) break;
          mbar_expect_tx(full(s), sbytes);
          const uint32_t dst = sD + (uint32_t)s * sbytes;
          if constexpr (KS::split) {  // 3D boxes {64, rows, 2}: the hi tile, then the lo tile, of data and V
            tma_load_3d(dst, &tmX, kt * KS::tile, tile * kTileRows, 0, full(s));
            tma_load_3d(dst + 2u * kStageBytes, &tmW, kt * KS::tile, 0, 0, full(s));
          } else {
            tma_load_2d(dst, &tmX, kt * KS::tile, tile * kTileRows, full(s));
            if (a.wstream) tma_load_2d(dst + kStageBytes, &tmW, kt * KS::tile, 0, full(s));
          }
        }
      }
      // drain: every issued load has completed before the CTA may exit
      if (*abort_flag) {
        for (int j = (it > NS ? it - NS : 0); j < it; ++j) {
          const unsigned long long t0 = gtimer();
          while (!mbar_try_wait(full(j % NS), (uint32_t)((j / NS) & 1)) && gtimer() - t0 < kWaitLimitNs) {
          }
        }
        const unsigned long long t0 = gtimer();
        while (!a.wstream && !mbar_try_wait(vbar, 0) && gtimer() - t0 < kWaitLimitNs) {
        }
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issuer
      constexpr uint32_t fmt = KS::tf32 ? 2u : (std::is_same<InT, __half>::value ? 0u : 1u);
      const uint32_t idesc = (FORM == 1) ? idesc_f16kind(128, a.Np, fmt) : idesc_f16kind(128, 128, fmt);
      // Shared-memory descriptors: the address field holds address / 16 in its low 14 bits (shared memory
      // is below 256 KB, so offsets add without a carry out of the field); a 16-element K step is +2.
      // The issue loop is kept short: one thread issuing small MMAs is otherwise slower than the tensor
      // pipe executing them.
      const unsigned long long dX0 = sw128_desc(sD), dV0 = sw128_desc(sV);
      const uint32_t vkt = (uint32_t)(a.VR * 128) >> 4;  // one 64-wide K tile of V
      const bool two_mb = (FORM != 1) && a.MB > 1;       // second 128-row block of V (form 2)
      bool ok = a.wstream ? true : wait_bounded(vbar, 0, ab);
      int it = 0, tcount = 0;
      for (int tile = blockIdx.x; ok && tile < ntiles; tile += gridDim.x, ++tcount) {
        const int b = tcount & 1;
        if (!(ok = wait_bounded(tempty(b), (uint32_t)(((tcount >> 1) & 1) ^ 1), ab))) break;
        tc_fence_after();
        const uint32_t dacc = tmem + (uint32_t)(b * a.acc_cols);
        for (int kt = 0; kt < a.KT; ++kt, ++it) {
          const int s = it % NS;
          if (!(ok = wait_bounded(full(s), (uint32_t)((it / NS) & 1), ab))) break;
          tc_fence_after();
          const unsigned long long xd = dX0 + (uint32_t)s * (sbytes >> 4);
          // a streamed eigenbasis tile follows the data tile(s) of the stage
          const uint32_t voff = (uint32_t)((KS::split ? 2 : 1) * kStageBytes) >> 4;
          const unsigned long long vd = a.wstream ? xd + voff : dV0 + (uint32_t)kt * vkt;
          // split form: lo planes one data tile / one eigenbasis tile (VR rows) after the hi planes
          const uint32_t xlo = (uint32_t)kStageBytes >> 4, vlo = (uint32_t)(a.VR * 128) >> 4;
          const int nk = min(4, (a.C - kt * KS::tile + KS::step - 1) / KS::step);  // K steps inside C
          auto mma = [&](uint32_t d, unsigned long long ad, unsigned long long bd, uint32_t acc) {
            if constexpr (KS::tf32) tc_mma_tf32(d, ad, bd, idesc, acc);
            else tc_mma(d, ad, bd, idesc, acc);
          };
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            if (kk < nk) {
              const uint32_t accum = (kt > 0 || kk > 0) ? 1u : 0u;
              if (FORM == 1) {
                mma(dacc, xd + 2u * kk, vd + 2u * kk, accum);
                if constexpr (KS::split) {
                  mma(dacc, xd + xlo + 2u * kk, vd + 2u * kk, 1u);
                  mma(dacc, xd + 2u * kk, vd + vlo + 2u * kk, 1u);
                }
              } else {
                mma(dacc, vd + 2u * kk, xd + 2u * kk, accum);
                if constexpr (KS::split) {
                  mma(dacc, vd + 2u * kk, xd + xlo + 2u * kk, 1u);
                  mma(dacc, vd + vlo + 2u * kk, xd + 2u * kk, 1u);
                }
                if (two_mb) {
                  const unsigned long long v1 = vd + (uint32_t)(kStageBytes >> 4);  // rows 128.. of the tile
                  mma(dacc + 128u, v1 + 2u * kk, xd + 2u * kk, accum);
                  if constexpr (KS::split) {
                    mma(dacc + 128u, v1 + 2u * kk, xd + xlo + 2u * kk, 1u);
                    mma(dacc + 128u, v1 + vlo + 2u * kk, xd + 2u * kk, 1u);
                  }
                }
              }
            }
          }
          tc_commit(empty(s));
        }
        if (!ok) break;
        tc_commit(tfull(b));
      }
      // all MMAs issued by this thread are complete once `drain` fires
      tc_commit(drain);
      const unsigned long long t0 = gtimer();
      while (!mbar_try_wait(drain, 0) && gtimer() - t0 < kWaitLimitNs) {
      }
    }
    __syncwarp();
  } else if (warp == TcWarps<FINAL>::rwarp) {
    // ---------------- TMA of R~ (last pass): 16-column chunks of the tile's 128 rows.  Chunk ci belongs to
    // epilogue half ci % 2, which consumes its chunks in order from its own ring of kRHalf slots (a ring
    // shared by both halves would let one half run a phase ahead of a slot and read it early).  Slot s of
    // half hh is hh * kRHalf + s, s < a.rhalf; its bytes sit at ring position hh * a.rhalf + s.
    if (rtma && lane == 0) {
      asm volatile("griddepcontrol.wait;" ::: "memory");
      const int nchunk = (a.Np + 15) / 16;
      const int Jh[2] = {(nchunk + 1) / 2, nchunk / 2};  // chunks per tile of each half
      int issued[2] = {0, 0};
      bool ok = true;
      int tcnt = 0;
      for (int tile = blockIdx.x; ok && tile < ntiles; tile += gridDim.x, ++tcnt) {
        for (int ci = 0; ci < nchunk; ++ci) {
          const int hh = ci & 1;
          const int k = tcnt * Jh[hh] + (ci >> 1);
          const int slot = hh * kRHalf + (k % a.rhalf);
          if (!(ok = wait_bounded(rempty(slot), (uint32_t)(((k / a.rhalf) & 1) ^ 1), ab))) break;
          mbar_expect_tx(rfull(slot), kRBytes);
          tma_load_2d(sR + (uint32_t)(hh * a.rhalf + k % a.rhalf) * kRBytes, &tmR, ci * 16, tile * kTileRows,
                      rfull(slot));
          issued[hh] = k + 1;
        }
      }
      if (!ok) {  // every issued load completes before the CTA may exit
        for (int hh = 0; hh < 2; ++hh)
          for (int k = (issued[hh] > a.rhalf ? issued[hh] - a.rhalf : 0); k < issued[hh]; ++k) {
            const unsigned long long t0 = gtimer();
            while (!mbar_try_wait(rfull(hh * kRHalf + (k % a.rhalf)), (uint32_t)((k / a.rhalf) & 1)) &&
                   gtimer() - t0 < kWaitLimitNs) {
            }
          }
      }
    }
    __syncwarp();
  } else if (warp >= 2) {
    // ---------------- epilogue: NG warps per TMEM lane quadrant, each taking every NG-th 16-column chunk
    constexpr int NG = TcWarps<FINAL>::groups;
    const int q = warp & 3;          // TMEM lane quadrant this warp may access
    const int h = (warp - 2) >> 2;   // which share of the column chunks
    // TMA store of one [32][16] box from this warp's two staging buffers (used alternately; a buffer is
    // rewritten once the store issued from it two boxes earlier has finished reading it)
    const uint32_t sOw = sO + (uint32_t)(warp - 2) * 2u * kOBytes;
    int ocnt = 0;
    auto emit = [&](const float (&v)[16], int x0, int x1, int x2) {
      const uint32_t buf = sOw + (uint32_t)(ocnt & 1) * kOBytes;
      if (ocnt >= 2) {
        if (lane == 0) asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
        __syncwarp();
      }
      stage_row<StageT>(buf, lane, v);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic writes -> async-proxy reads
      __syncwarp();
      if (lane == 0) {
        if (FORM == 1) tma_store_2d(&tmO, buf, x0, x1);
        else tma_store_3d(&tmO, buf, x0, x1, x2);
        asm volatile("cp.async.bulk.commit_group;" ::: "memory");
      }
      ++ocnt;
    };
    int tcount = 0;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++tcount) {
      const int b = tcount & 1;
      if (!wait_bounded(tfull(b), (uint32_t)((tcount >> 1) & 1), ab)) break;
      tc_fence_after();
      const uint32_t tacc = tmem + (uint32_t)(b * a.acc_cols) + ((uint32_t)(q * 32) << 16);
      const int row0 = tile * kTileRows;
      if (FORM == 1) {
        // one thread per row; its 16 consecutive output columns are contiguous in memory (oc == 1).
        // This warp takes the 16-column chunks c0 = h*16 + 16*NG*j.  The TMEM load of chunk j+1 is
        // issued before chunk j is processed; in the last pass the residual R of chunk j+2 is
        // fetched while chunk j is processed.
        const int r = row0 + q * 32 + lane;
        const bool valid = r < a.rows;
        const int ia = valid ? r / a.B : 0;
        const int ib = valid ? r - ia * a.B : 0;
        const long long obase = (long long)ia * a.oa + (long long)ib * a.ob;
        const float sab = (a.scale && valid) ? a.lamA[ia] + a.lamB[ib] : 0.0f;
        const bool null_row = a.singular && ia == 0 && ib == 0;
        const float zs = (a.last && a.shift_src) ? ldexpf(1.0f, a.sG - *a.shift_src) : 1.0f;
        const bool vec = a.vec && valid;
        const int J = (a.Np - h * 16 + 16 * NG - 1) / (16 * NG);  // chunks of this warp (warp-uniform)
        auto col = [&](int j) { return h * 16 + 16 * NG * j; };
        const int trow = q * 32 + lane;  // row within the tile
        // R~ chunk j of this warp staged by TMA: wait for it, read this row's 16 values (32-byte swizzle:
        // 16-byte piece i of row r sits at piece i ^ ((r / 4) % 2)), release the slot.
        auto take_r = [&](int j, uint4 (&rb)[2]) {
          const int k = tcount * J + j;  // this half's chunk sequence number
          const int slot = h * kRHalf + (k % a.rhalf);
          if (!wait_bounded(rfull(slot), (uint32_t)((k / a.rhalf) & 1), ab)) return false;
          const uint32_t base = sR + (uint32_t)(h * a.rhalf + k % a.rhalf) * kRBytes + (uint32_t)trow * 32u;
#pragma unroll
          for (int i = 0; i < 2; ++i) {
            uint4 w;
            asm volatile("ld.shared.v4.b32 {%0, %1, %2, %3}, [%4];"
                         : "=r"(w.x), "=r"(w.y), "=r"(w.z), "=r"(w.w)
                         : "r"(base + (uint32_t)((i ^ ((trow >> 2) & 1)) << 4))
                         : "memory");
            rb[i] = w;
          }
          // the slot is next written by TMA (async proxy): order these generic-proxy reads before it
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          mbar_arrive(rempty(slot));
          return true;
        };
        auto fetch_r = [&](int j, uint4 (&rb)[2]) {
          if (FINAL && !KS::tf32 && !KS::split && !rtma && vec && j < J && col(j) + 16 <= a.Cout) {
            const uint4* rp = reinterpret_cast<const uint4*>(a.Rt + (long long)r * a.rpitch + col(j));
            rb[0] = __ldg(rp);
            rb[1] = __ldg(rp + 1);
          }
        };
        auto process = [&](int c0, const uint32_t (&t)[16], const uint4 (&rcur)[2]) {
          if (!valid && !a.tstore) return;
          float v[16];
#pragma unroll
          for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(t[i]);
          if (a.scale) {  // Algorithm 7, Hadamard step: multiply by G = 1 / (lam_a + lam_b + lam_c)
            const float4* lc4 = reinterpret_cast<const float4*>(a.lamC + c0);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
              const float4 l = __ldg(lc4 + i);
              v[4 * i + 0] *= rcp_approx(sab + l.x) * a.gscale;
              v[4 * i + 1] *= rcp_approx(sab + l.y) * a.gscale;
              v[4 * i + 2] *= rcp_approx(sab + l.z) * a.gscale;
              v[4 * i + 3] *= rcp_approx(sab + l.w) * a.gscale;
            }
            if (null_row && c0 == 0) v[0] = 0.0f;
          }
          if (a.last) {
#pragma unroll
            for (int j = 0; j < 16; ++j) v[j] *= zs;
          } else if constexpr (KS::tf32) {  // intermediates: round to TF32 (nearest even) for the next pass
#pragma unroll
            for (int j = 0; j < 16; ++j) v[j] = tf32_rn(v[j]);
          }
          if (a.tstore) emit(v, c0, row0 + q * 32, 0);  // rows past `rows`, columns past Cout: clipped
          if (!valid) return;
          if (vec && c0 + 16 <= a.Cout) {
            if (!a.tstore) store16<OutT>(a.out, a.oplane, obase + c0, v);
            if (FINAL && KS::split) {  // R~ = hi + lo, 16 values of this row from each plane
              const uint4* hp = reinterpret_cast<const uint4*>(a.Rt + (long long)r * a.rpitch + c0);
              const uint4* lq = reinterpret_cast<const uint4*>(Rlo + (long long)r * a.rpitch + c0);
              const uint4 h0 = __ldg(hp), h1 = __ldg(hp + 1), l0 = __ldg(lq), l1 = __ldg(lq + 1);
              const uint32_t hw[8] = {h0.x, h0.y, h0.z, h0.w, h1.x, h1.y, h1.z, h1.w};
              const uint32_t lw[8] = {l0.x, l0.y, l0.z, l0.w, l1.x, l1.y, l1.z, l1.w};
              float d0 = 0.0f, d1 = 0.0f;
#pragma unroll
              for (int i = 0; i < 8; ++i) {
                const float2 rh = lp2_to_f32<__nv_bfloat16>(hw[i]), rl = lp2_to_f32<__nv_bfloat16>(lw[i]);
                d0 = fmaf((rh.x + rl.x) * rs, v[2 * i], d0);
                d1 = fmaf((rh.y + rl.y) * rs, v[2 * i + 1], d1);
                zmax = fmaxf(zmax, fmaxf(fabsf(v[2 * i]), fabsf(v[2 * i + 1])));
              }
              red0.add(d0 + d1);
              red1.add(((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7])) +
                       (((v[8] + v[9]) + (v[10] + v[11])) + ((v[12] + v[13]) + (v[14] + v[15]))));
            } else if (FINAL && KS::tf32) {  // R~ in FP32 containers, 16 values of this row
              const float4* rp =
                  reinterpret_cast<const float4*>(reinterpret_cast<const float*>(a.Rt) + (long long)r * a.rpitch + c0);
              float d0 = 0.0f, d1 = 0.0f;
#pragma unroll
              for (int i = 0; i < 4; ++i) {
                const float4 rr = __ldg(rp + i);
                d0 = fmaf(rr.x * rs, v[4 * i], fmaf(rr.y * rs, v[4 * i + 1], d0));
                d1 = fmaf(rr.z * rs, v[4 * i + 2], fmaf(rr.w * rs, v[4 * i + 3], d1));
                zmax = fmaxf(zmax, fmaxf(fmaxf(fabsf(v[4 * i]), fabsf(v[4 * i + 1])),
                                         fmaxf(fabsf(v[4 * i + 2]), fabsf(v[4 * i + 3]))));
              }
              red0.add(d0 + d1);
              red1.add(((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7])) +
                       (((v[8] + v[9]) + (v[10] + v[11])) + ((v[12] + v[13]) + (v[14] + v[15]))));
            } else if constexpr (FINAL && !KS::split) {
              const uint32_t rw[8] = {rcur[0].x, rcur[0].y, rcur[0].z, rcur[0].w,
                                      rcur[1].x, rcur[1].y, rcur[1].z, rcur[1].w};
              float d0 = 0.0f, d1 = 0.0f;
#pragma unroll
              for (int i = 0; i < 8; ++i) {
                const float2 rr = lp2_to_f32<InT>(rw[i]);
                d0 = fmaf(rr.x * rs, v[2 * i], d0);
                d1 = fmaf(rr.y * rs, v[2 * i + 1], d1);
                zmax = fmaxf(zmax, fmaxf(fabsf(v[2 * i]), fabsf(v[2 * i + 1])));
              }
              red0.add(d0 + d1);
              red1.add(((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7])) +
                       (((v[8] + v[9]) + (v[10] + v[11])) + ((v[12] + v[13]) + (v[14] + v[15]))));
            }
          } else {
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              const int c = c0 + j;
              if (c < a.Cout) {
                const long long o = obase + (long long)c * a.oc;
                if (!a.tstore) store_out<OutT>(a.out, a.oplane, o, v[j]);
                if (FINAL) {
                  float rv;
                  if constexpr (KS::tf32) rv = __ldg(reinterpret_cast<const float*>(a.Rt) + (long long)r * a.rpitch + c);
                  else if constexpr (KS::split)
                    rv = lp2_to_f32<__nv_bfloat16>(__ldg(a.Rt + (long long)r * a.rpitch + c)).x +
                         lp2_to_f32<__nv_bfloat16>(__ldg(Rlo + (long long)r * a.rpitch + c)).x;
                  else rv = lp2_to_f32<InT>(__ldg(a.Rt + (long long)r * a.rpitch + c)).x;
                  red0.add(rv * rs * v[j]);
                  red1.add(v[j]);
                  zmax = fmaxf(zmax, fabsf(v[j]));
                }
              }
            }
          }
        };
        uint32_t tA[16], tB[16];
        uint4 rA[2], rB[2];
        if (rtma) {
          bool ok = true;
          for (int j = 0; ok && j < J; ++j) {
            tc_ld16_issue(tacc + (uint32_t)col(j), tA);
            ok = __all_sync(0xffffffffu, take_r(j, rA));  // warp-uniform: tcgen05.ld is .sync.aligned
            tc_ld16_wait(tA);
            if (ok) process(col(j), tA, rA);
          }
        } else {
          if (J > 0) {
            tc_ld16_issue(tacc + (uint32_t)col(0), tA);
            fetch_r(0, rA);
            fetch_r(1, rB);
            tc_ld16_wait(tA);
          }
          for (int j = 0; j < J; j += 2) {
            if (j + 1 < J) tc_ld16_issue(tacc + (uint32_t)col(j + 1), tB);
            process(col(j), tA, rA);
            fetch_r(j + 2, rA);
            if (j + 1 < J) {
              tc_ld16_wait(tB);
              if (j + 2 < J) tc_ld16_issue(tacc + (uint32_t)col(j + 2), tA);
              process(col(j + 1), tB, rB);
              fetch_r(j + 3, rB);
              if (j + 2 < J) tc_ld16_wait(tA);
            }
          }
        }
      } else {
        // one thread per output index; its 16 consecutive rows are contiguous in memory (ob == 1).
        // Chunks (M-block mb, rows c0 = h*16 + 16*NG*j) in a fixed order, TMEM loads one chunk ahead.
        const int per_mb = (kTileRows - h * 16 + 16 * NG - 1) / (16 * NG);
        const int J = a.MB * per_mb;
        auto taddr = [&](int j) {
          const int mb = j / per_mb, c0 = h * 16 + 16 * NG * (j - mb * per_mb);
          return tacc + (uint32_t)(mb * 128 + c0);
        };
        auto process = [&](int j, const uint32_t (&t)[16]) {
          const int mb = j / per_mb, c0 = h * 16 + 16 * NG * (j - mb * per_mb);
          const int cb = mb * 128 + q * 32;
          const int c = cb + lane;
          const int r0 = row0 + c0;
          if (r0 >= a.rows) return;  // warp-uniform
          float v[16];
#pragma unroll
          for (int i = 0; i < 16; ++i) v[i] = KS::tf32 ? tf32_rn(__uint_as_float(t[i])) : __uint_as_float(t[i]);
          int ia = r0 / a.B;
          int ib = r0 - ia * a.B;
          if (a.tstore) {  // B % 16 == 0: the 16 rows share one a; output indices past Cout are clipped
            if (a.tperm) emit(v, ib, ia, cb);
            else emit(v, ib, cb, ia);
            return;
          }
          if (c >= a.Cout) return;
          if (a.vec && ib + 16 <= a.B && r0 + 16 <= a.rows) {
            store16<OutT>(a.out, a.oplane, (long long)ia * a.oa + ib + (long long)c * a.oc, v);
          } else {
#pragma unroll
            for (int i = 0; i < 16; ++i) {
              if (r0 + i < a.rows)
                store_out<OutT>(a.out, a.oplane, (long long)ia * a.oa + (long long)ib * a.ob + (long long)c * a.oc, v[i]);
              if (++ib == a.B) {
                ib = 0;
                ++ia;
              }
            }
          }
        };
        uint32_t tA[16], tB[16];
        if (J > 0) {
          tc_ld16_issue(taddr(0), tA);
          tc_ld16_wait(tA);
        }
        for (int j = 0; j < J; j += 2) {
          if (j + 1 < J) tc_ld16_issue(taddr(j + 1), tB);
          process(j, tA);
          if (j + 1 < J) {
            tc_ld16_wait(tB);
            if (j + 2 < J) tc_ld16_issue(taddr(j + 2), tA);
            process(j + 1, tB);
            if (j + 2 < J) tc_ld16_wait(tA);
          }
        }
      }
      tc_fence_before();
      mbar_arrive(tempty(b));
    }
    // this warp's TMA stores are complete before the CTA may exit
    if (lane == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
  }

  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)a.tmem_cols)
                 : "memory");
  }
  if constexpr (FINAL) {
    // max |Z| of the block -> one atomicMax (order-independent, so deterministic)
    __shared__ float smax[TcWarps<FINAL>::threads / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) zmax = fmaxf(zmax, __shfl_xor_sync(0xffffffffu, zmax, o));
    if (lane == 0) smax[warp] = zmax;
    __syncthreads();
    if (threadIdx.x == 0) {
      float m = 0.0f;
      for (int w = 0; w < TcWarps<FINAL>::threads / 32; ++w) m = fmaxf(m, smax[w]);
      atomicMax(&a.st->zmax_bits, __float_as_uint(m));
    }
    double acc[2] = {acc_value(red0), acc_value(red1)};
    SolveState* st = a.st;
    const long long N = a.N;
    grid_reduce<2>(acc, a.partials, &st->tickets[kTkPrec], gridDim.x, blockIdx.x,
                   [st, N, shR](const double(&s)[2]) {
                     st->zmax = __uint_as_float(atomicExch(&st->zmax_bits, 0u));
                     const double v[2] = {ldexp(s[0], -shR), s[1]};
                     if (!st->timeout) {
                       fin_precond(st, N, v);
                       plan_next_direction(st);
                     } else {
                       st->status = TPCG_ERR_TIMEOUT;
                       st->done = 1;
                     }
                   });
  }
}

// ------------------------------------------------------------------ fused pair of passes
// In Algorithm 7 the Hadamard step by G sits between the forward and the
// backward mode product along one axis.  When that axis is the contiguous
// index of the forward pass's input, both products contract it over the same
// 128-row tiles, so one kernel runs the two with the scaled intermediate of a
// tile held in shared memory (it is neither written out nor read back):
//   stage 1 (form 1): D1[row][c'] = X[row][:] . W1^T[c'][:], times G and the
//            FP16 range factor, rounded to FP16/BF16 into T[row][c'] (K-major,
//            128-byte swizzle: the layout TMA gives a loaded operand);
//   stage 2 (form 2): D2[c][row] = W2^T[c][:] . T[row][:], stored in the
//            backward pass's output layout.
// Stage 1 issues the MMAs of the forward pass and stage 2 those of the
// backward pass, in the same order, and the intermediate takes the same G
// product and the same rounding: the output is bitwise that of the two passes.
// Warps: 0 TMA, 1 MMA (stage 1 of tile i+1 is issued before stage 2 of tile
// i), 2..17 epilogue, software-pipelined: stage 1 of tile i, then stage 2 of
// tile i-1, so that the tensor core runs stage 2 of tile i-1 while the
// epilogue scales tile i.  TMEM: D1 and D2 double-buffered, 4 x 128 columns;
// T double-buffered: the epilogue writes T for tile i after it has seen stage
// 2 of tile i-2 complete.
constexpr int kPairEpi = 16;
constexpr int kPairThreads = (2 + kPairEpi) * 32;
constexpr int kTBytes = kTileRows * 128;  // one 64-column K tile of T

template <class InT>
__global__ void __launch_bounds__(kPairThreads, 1)
    k_modeprod_pair(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmW1,
                    const __grid_constant__ CUtensorMap tmW2, const __grid_constant__ CUtensorMap tmO, TcArgs a) {
  if (a.st && a.st->done) return;
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t* sm = smem_raw + (base - raw);
  const int KT = a.KT, NS = a.NS;
  const uint32_t sW1 = base;
  const uint32_t sW2 = sW1 + (uint32_t)KT * a.VR * 128u;  // VR % 8 == 0: 1024-aligned
  const uint32_t sT = sW2 + (uint32_t)KT * 128u * 128u;  // two buffers of KT K tiles
  const uint32_t sD = sT + 2u * (uint32_t)KT * kTBytes;
  const uint32_t sO = sD + (uint32_t)NS * kStageBytes;
  constexpr uint32_t kOBytes = 32u * 16u * (uint32_t)sizeof(InT);
  uint8_t* barp = sm + (sO - base) + (size_t)kPairEpi * 2 * kOBytes;
  const uint32_t bars = smem_u32(barp);
  auto full = [&](int s) { return bars + 8u * s; };
  auto empty = [&](int s) { return bars + 8u * (NS + s); };
  auto d1full = [&](int b) { return bars + 8u * (2 * NS + b); };
  auto d1empty = [&](int b) { return bars + 8u * (2 * NS + 2 + b); };
  auto d2full = [&](int b) { return bars + 8u * (2 * NS + 4 + b); };
  auto d2empty = [&](int b) { return bars + 8u * (2 * NS + 6 + b); };
  auto tready = [&](int b) { return bars + 8u * (2 * NS + 8 + b); };
  const uint32_t vbar = bars + 8u * (2 * NS + 10);
  const uint32_t drain = bars + 8u * (2 * NS + 11);
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(barp + 8 * (2 * NS + 12));
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_holder + 1);
  const Abort ab{abort_flag, a.err, a.st};

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < NS; ++s) {
      mbar_init(full(s), 1);
      mbar_init(empty(s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(d1full(b), 1);
      mbar_init(d1empty(b), kPairEpi * 32);
      mbar_init(d2full(b), 1);
      mbar_init(d2empty(b), kPairEpi * 32);
      mbar_init(tready(b), kPairEpi * 32);
    }
    mbar_init(vbar, 1);
    mbar_init(drain, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_holder)),
                 "r"(512u)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_holder;
  const int ntiles = (a.rows + kTileRows - 1) / kTileRows;
  const int nmine = ntiles > (int)blockIdx.x ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer: both eigenbases once, then the K tiles of every row tile
      mbar_expect_tx(vbar, (uint32_t)KT * (uint32_t)(a.VR + 128) * 128u);
      for (int kt = 0; kt < KT; ++kt) tma_load_2d(sW1 + (uint32_t)kt * a.VR * 128u, &tmW1, kt * kKTile, 0, vbar);
      for (int kt = 0; kt < KT; ++kt) tma_load_2d(sW2 + (uint32_t)kt * 128u * 128u, &tmW2, kt * kKTile, 0, vbar);
      asm volatile("griddepcontrol.wait;" ::: "memory");
      int it = 0;
      for (int i = 0; i < nmine && !*abort_flag; ++i) {
        const int tile = (int)blockIdx.x + i * (int)gridDim.x;
        for (int kt = 0; kt < KT; ++kt, ++it) {
          const int s = it % NS;
          if (!wait_bounded(empty(s), (uint32_t)(((it / NS) & 1) ^ 1), ab)) break;
          mbar_expect_tx(full(s), kStageBytes);
          tma_load_2d(sD + (uint32_t)s * kStageBytes, &tmX, kt * kKTile, tile * kTileRows, full(s));
        }
      }
      if (*abort_flag) {  // every issued load completes before the CTA may exit
        for (int j = (it > NS ? it - NS : 0); j < it; ++j) {
          const unsigned long long t0 = gtimer();
          while (!mbar_try_wait(full(j % NS), (uint32_t)((j / NS) & 1)) && gtimer() - t0 < kWaitLimitNs) {
          }
        }
        const unsigned long long t0 = gtimer();
        while (!mbar_try_wait(vbar, 0) && gtimer() - t0 < kWaitLimitNs) {
        }
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issuer
      constexpr uint32_t fmt = std::is_same<InT, __half>::value ? 0u : 1u;
      const uint32_t idesc1 = idesc_f16kind(128, a.Np, fmt), idesc2 = idesc_f16kind(128, 128, fmt);
      const unsigned long long dX0 = sw128_desc(sD), dW1 = sw128_desc(sW1), dW2 = sw128_desc(sW2), dT = sw128_desc(sT);
      const uint32_t w1kt = (uint32_t)(a.VR * 128) >> 4, w2kt = (uint32_t)(128 * 128) >> 4,
                     tkt = (uint32_t)kTBytes >> 4;
      bool ok = wait_bounded(vbar, 0, ab);
      int it = 0;
      auto stage1 = [&](int i) {  // forward product of tile i into D1[i & 1]
        const int b = i & 1;
        if (!wait_bounded(d1empty(b), (uint32_t)(((i >> 1) & 1) ^ 1), ab)) return false;
        tc_fence_after();
        const uint32_t dacc = tmem + (uint32_t)(b * 128);
        for (int kt = 0; kt < KT; ++kt, ++it) {
          const int s = it % NS;
          if (!wait_bounded(full(s), (uint32_t)((it / NS) & 1), ab)) return false;
          tc_fence_after();
          const unsigned long long xd = dX0 + (uint32_t)s * (uint32_t)(kStageBytes >> 4);
          const unsigned long long wd = dW1 + (uint32_t)kt * w1kt;
          const int nk = min(4, (a.C - kt * kKTile + 15) >> 4);
#pragma unroll
          for (int kk = 0; kk < 4; ++kk)
            if (kk < nk) tc_mma(dacc, xd + 2u * kk, wd + 2u * kk, idesc1, (kt > 0 || kk > 0) ? 1u : 0u);
          tc_commit(empty(s));
        }
        tc_commit(d1full(b));
        return true;
      };
      auto stage2 = [&](int i) {  // backward product of tile i (T in shared memory) into D2[i & 1]
        const int b = i & 1;
        if (!wait_bounded(tready(b), (uint32_t)((i >> 1) & 1), ab)) return false;
        if (!wait_bounded(d2empty(b), (uint32_t)(((i >> 1) & 1) ^ 1), ab)) return false;
        tc_fence_after();
        const uint32_t dacc = tmem + 256u + (uint32_t)(b * 128);
        for (int kt = 0; kt < KT; ++kt) {
          const unsigned long long wd = dW2 + (uint32_t)kt * w2kt, td = dT + (uint32_t)(b * KT + kt) * tkt;
          const int nk = min(4, (a.C - kt * kKTile + 15) >> 4);
#pragma unroll
          for (int kk = 0; kk < 4; ++kk)
            if (kk < nk) tc_mma(dacc, wd + 2u * kk, td + 2u * kk, idesc2, (kt > 0 || kk > 0) ? 1u : 0u);
        }
        tc_commit(d2full(b));
        return true;
      };
      if (ok && nmine > 0) ok = stage1(0);
      for (int i = 0; ok && i < nmine; ++i) {
        if (i + 1 < nmine && !(ok = stage1(i + 1))) break;
        ok = stage2(i);
      }
      tc_commit(drain);  // every MMA this thread issued is complete once `drain` fires
      const unsigned long long t0 = gtimer();
      while (!mbar_try_wait(drain, 0) && gtimer() - t0 < kWaitLimitNs) {
      }
    }
    __syncwarp();
  } else if (warp >= 2) {
    // ---------------- epilogue: four warps per TMEM lane quadrant, warp h of a quadrant taking the 16-column
    // chunks h*16 + 64*j
    const int q = warp & 3, h = (warp - 2) >> 2;
    const int trow = q * 32 + lane;
    const uint32_t sOw = sO + (uint32_t)(warp - 2) * 2u * kOBytes;
    int ocnt = 0;
    auto emit = [&](const float (&v)[16], int x0, int x1, int x2) {  // as in k_modeprod_tc, form 2
      const uint32_t buf = sOw + (uint32_t)(ocnt & 1) * kOBytes;
      if (ocnt >= 2) {
        if (lane == 0) asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
        __syncwarp();
      }
      stage_row<InT>(buf, lane, v);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) {
        tma_store_3d(&tmO, buf, x0, x1, x2);
        asm volatile("cp.async.bulk.commit_group;" ::: "memory");
      }
      ++ocnt;
    };
    const int J1 = (a.Np - h * 16 + 63) / 64;  // stage-1 chunks of this warp (at most 2)
    // stage 1 of tile i: T[b][row][c'] = round(D1[row][c'] * G(row, c') * 2^-sG)
    auto epi1 = [&](int i) {
      const int tile = (int)blockIdx.x + i * (int)gridDim.x;
      const int b = i & 1;
      const int r = tile * kTileRows + trow;
      const bool valid = r < a.rows;
      const int ia = valid ? r / a.B1 : 0;
      const int ib = valid ? r - ia * a.B1 : 0;
      const float sab = valid ? a.lamA[ia] + a.lamB[ib] : 0.0f;
      const bool null_row = a.singular && ia == 0 && ib == 0;
      if (!__all_sync(0xffffffffu, wait_bounded(d1full(b), (uint32_t)((i >> 1) & 1), ab))) return false;
      tc_fence_after();
      const uint32_t tacc = tmem + (uint32_t)(b * 128) + ((uint32_t)(q * 32) << 16);
      uint32_t t0[16], t1[16];
      if (J1 > 0) tc_ld16_issue(tacc + (uint32_t)(h * 16), t0);
      if (J1 > 1) tc_ld16_issue(tacc + (uint32_t)(h * 16 + 64), t1);
      if (J1 > 0) tc_ld16_wait(t0);
      if (J1 > 1) tc_ld16_wait(t1);
      tc_fence_before();
      mbar_arrive(d1empty(b));
      const uint32_t tb = sT + (uint32_t)(b * KT) * (uint32_t)kTBytes;
      auto put = [&](int c0, const uint32_t (&t)[16]) {
        float v[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) v[k] = __uint_as_float(t[k]);
        const float4* lc4 = reinterpret_cast<const float4*>(a.lamC + c0);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const float4 l = __ldg(lc4 + k);
          v[4 * k + 0] *= rcp_approx(sab + l.x) * a.gscale;
          v[4 * k + 1] *= rcp_approx(sab + l.y) * a.gscale;
          v[4 * k + 2] *= rcp_approx(sab + l.z) * a.gscale;
          v[4 * k + 3] *= rcp_approx(sab + l.w) * a.gscale;
        }
        if (null_row && c0 == 0) v[0] = 0.0f;
        uint32_t pk[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          if constexpr (std::is_same<InT, __half>::value) {
            __half2 h2 = __floats2half2_rn(v[2 * k], v[2 * k + 1]);
            pk[k] = valid ? *reinterpret_cast<uint32_t*>(&h2) : 0u;
          } else {
            __nv_bfloat162 h2 = __floats2bfloat162_rn(v[2 * k], v[2 * k + 1]);
            pk[k] = valid ? *reinterpret_cast<uint32_t*>(&h2) : 0u;
          }
        }
        // 128-byte swizzle: 16-byte piece p of row trow sits at piece p ^ (trow % 8)
        const uint32_t rowa = tb + (uint32_t)(c0 >> 6) * (uint32_t)kTBytes + (uint32_t)trow * 128u;
        const uint32_t p0 = (uint32_t)((c0 & 63) >> 3);
#pragma unroll
        for (int k = 0; k < 2; ++k)
          asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(rowa + (((p0 + k) ^ (uint32_t)(trow & 7)) << 4)),
                       "r"(pk[4 * k]), "r"(pk[4 * k + 1]), "r"(pk[4 * k + 2]), "r"(pk[4 * k + 3])
                       : "memory");
      };
      if (J1 > 0) put(h * 16, t0);
      if (J1 > 1) put(h * 16 + 64, t1);
      // generic-proxy writes of T -> the tensor core's (async-proxy) reads
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_arrive(tready(b));
      return true;
    };
    // stage 2 of tile i: thread = output index c = q*32 + lane, chunk = 16 consecutive rows
    auto epi2 = [&](int i) {
      const int tile = (int)blockIdx.x + i * (int)gridDim.x;
      const int b = i & 1;
      const int row0 = tile * kTileRows;
      if (!__all_sync(0xffffffffu, wait_bounded(d2full(b), (uint32_t)((i >> 1) & 1), ab))) return false;
      tc_fence_after();
      const uint32_t tacc = tmem + 256u + (uint32_t)(b * 128) + ((uint32_t)(q * 32) << 16);
      uint32_t t0[16], t1[16];
      tc_ld16_issue(tacc + (uint32_t)(h * 16), t0);
      tc_ld16_issue(tacc + (uint32_t)(h * 16 + 64), t1);
      tc_ld16_wait(t0);
      tc_ld16_wait(t1);
      tc_fence_before();
      mbar_arrive(d2empty(b));
      const int cb = q * 32;
      auto out = [&](int c0, const uint32_t (&t)[16]) {
        const int r0 = row0 + c0;
        if (r0 >= a.rows || cb >= a.Cout) return;  // warp-uniform (rows % 16 == 0)
        float v[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) v[k] = __uint_as_float(t[k]);
        const int ia = r0 / a.B, ib = r0 - ia * a.B;
        if (a.tperm) emit(v, ib, ia, cb);
        else emit(v, ib, cb, ia);
      };
      out(h * 16, t0);
      out(h * 16 + 64, t1);
      return true;
    };
    bool ok = true;
    for (int i = 0; ok && i < nmine; ++i) {
      ok = epi1(i);
      if (ok && i > 0) ok = epi2(i - 1);
    }
    if (ok && nmine > 0) epi2(nmine - 1);
    if (lane == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
  }

  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512u) : "memory");
  }
}

// ------------------------------------------------------------------ host side
// Fused pair of passes, split BF16 form.  The same two products as
// k_modeprod_pair (Algorithm 7: forward product along one axis, Hadamard step
// by G, backward product along the same axis) on hi/lo BF16 pairs: each K step
// issues hi.hi, lo.hi and hi.lo into one FP32 accumulator in the order of the
// per-pass split kernel, the epilogue of stage 1 multiplies by G in FP32 and
// splits into hi = bf16(v), lo = bf16(v - hi) (T, both planes, K-major with
// the 128-byte swizzle), and stage 2 writes the backward pass's output planes
// with the per-pass kernel's stores: the output is bitwise that of the two
// split passes.  One split eigenbasis stays resident (64 KB at 128 points):
// the backward product's A operand W2[c][c'] = W1^T holds the values of the
// forward product's B operand W1[c'][c], so stage 2 reads W1's tiles as an
// MN-major operand (the two 64-row K tiles of W1 are its two 64-element M
// atoms).  T is double-buffered, as in k_modeprod_pair: the epilogue scales
// tile i while the tensor core runs stage 2 of tile i-1.
constexpr int kPairSplitEpi = 16;
constexpr int kPairSplitThreads = (2 + kPairSplitEpi) * 32;

__global__ void __launch_bounds__(kPairSplitThreads, 1)
    k_modeprod_pair_split(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmW1,
                          const __grid_constant__ CUtensorMap tmW2, TcArgs a) {
  if (a.st && a.st->done) return;
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t* sm = smem_raw + (base - raw);
  const int KT = a.KT, NS = a.NS;
  // per K tile: the hi tile, then the lo tile (one 3D TMA box {64, rows, 2})
  const uint32_t w1kt = 2u * (uint32_t)a.VR * 128u, tkt = 2u * (uint32_t)kTBytes;
  const uint32_t sW1 = base;
  const uint32_t sT = sW1 + (uint32_t)KT * w1kt;  // VR % 8 == 0: 1024-aligned; two buffers of KT K tiles
  const uint32_t sD = sT + 2u * (uint32_t)KT * tkt;
  const uint32_t sbytes = 2u * (uint32_t)kStageBytes;
  uint8_t* barp = sm + (sD - base) + (size_t)NS * sbytes;
  const uint32_t bars = smem_u32(barp);
  auto full = [&](int s) { return bars + 8u * s; };
  auto empty = [&](int s) { return bars + 8u * (NS + s); };
  auto d1full = [&](int b) { return bars + 8u * (2 * NS + b); };
  auto d1empty = [&](int b) { return bars + 8u * (2 * NS + 2 + b); };
  auto d2full = [&](int b) { return bars + 8u * (2 * NS + 4 + b); };
  auto d2empty = [&](int b) { return bars + 8u * (2 * NS + 6 + b); };
  auto tready = [&](int b) { return bars + 8u * (2 * NS + 8 + b); };
  const uint32_t vbar = bars + 8u * (2 * NS + 10);
  const uint32_t drain = bars + 8u * (2 * NS + 11);
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(barp + 8 * (2 * NS + 12));
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_holder + 1);
  const Abort ab{abort_flag, a.err, a.st};

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < NS; ++s) {
      mbar_init(full(s), 1);
      mbar_init(empty(s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(d1full(b), 1);
      mbar_init(d1empty(b), kPairSplitEpi * 32);
      mbar_init(d2full(b), 1);
      mbar_init(d2empty(b), kPairSplitEpi * 32);
      mbar_init(tready(b), kPairSplitEpi * 32);
    }
    mbar_init(vbar, 1);
    mbar_init(drain, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_holder)),
                 "r"(512u)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_holder;
  const int ntiles = (a.rows + kTileRows - 1) / kTileRows;
  const int nmine = ntiles > (int)blockIdx.x ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer: the split eigenbasis once, then the K tiles of every row tile
      mbar_expect_tx(vbar, (uint32_t)KT * w1kt);
      for (int kt = 0; kt < KT; ++kt) tma_load_3d(sW1 + (uint32_t)kt * w1kt, &tmW1, kt * kKTile, 0, 0, vbar);
      asm volatile("griddepcontrol.wait;" ::: "memory");
      int it = 0;
      for (int i = 0; i < nmine && !*abort_flag; ++i) {
        const int tile = (int)blockIdx.x + i * (int)gridDim.x;
        for (int kt = 0; kt < KT; ++kt, ++it) {
          const int s = it % NS;
          if (!wait_bounded(empty(s), (uint32_t)(((it / NS) & 1) ^ 1), ab)) break;
          mbar_expect_tx(full(s), sbytes);
          tma_load_3d(sD + (uint32_t)s * sbytes, &tmX, kt * kKTile, tile * kTileRows, 0, full(s));
        }
      }
      if (*abort_flag) {  // every issued load completes before the CTA may exit
        for (int j = (it > NS ? it - NS : 0); j < it; ++j) {
          const unsigned long long t0 = gtimer();
          while (!mbar_try_wait(full(j % NS), (uint32_t)((j / NS) & 1)) && gtimer() - t0 < kWaitLimitNs) {
          }
        }
        const unsigned long long t0 = gtimer();
        while (!mbar_try_wait(vbar, 0) && gtimer() - t0 < kWaitLimitNs) {
        }
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issuer (BF16 operands; the order of the per-pass split kernel)
      // stage 2: A (W1 read as W2) MN-major, transpose-A bit
      const uint32_t idesc1 = idesc_f16kind(128, a.Np, 1u), idesc2 = idesc_f16kind(128, 128, 1u) | (1u << 15);
      const unsigned long long dX0 = sw128_desc(sD), dW1 = sw128_desc(sW1), dT = sw128_desc(sT);
      // lo planes: one tile after the hi tile of the same K tile (descriptor units of 16 bytes)
      const uint32_t xlo = (uint32_t)kStageBytes >> 4, w1lo = (uint32_t)(a.VR * 128) >> 4,
                     tlo = (uint32_t)kTBytes >> 4;
      bool ok = wait_bounded(vbar, 0, ab);
      int it = 0;
      auto stage1 = [&](int i) {  // forward product of tile i into D1[i & 1]
        const int b = i & 1;
        if (!wait_bounded(d1empty(b), (uint32_t)(((i >> 1) & 1) ^ 1), ab)) return false;
        tc_fence_after();
        const uint32_t dacc = tmem + (uint32_t)(b * 128);
        for (int kt = 0; kt < KT; ++kt, ++it) {
          const int s = it % NS;
          if (!wait_bounded(full(s), (uint32_t)((it / NS) & 1), ab)) return false;
          tc_fence_after();
          const unsigned long long xd = dX0 + (uint32_t)s * (sbytes >> 4);
          const unsigned long long wd = dW1 + (uint32_t)kt * (w1kt >> 4);
          const int nk = min(4, (a.C - kt * kKTile + 15) >> 4);
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            if (kk < nk) {
              tc_mma(dacc, xd + 2u * kk, wd + 2u * kk, idesc1, (kt > 0 || kk > 0) ? 1u : 0u);
              tc_mma(dacc, xd + xlo + 2u * kk, wd + 2u * kk, idesc1, 1u);
              tc_mma(dacc, xd + 2u * kk, wd + w1lo + 2u * kk, idesc1, 1u);
            }
          }
          tc_commit(empty(s));
        }
        tc_commit(d1full(b));
        return true;
      };
      auto stage2 = [&](int i) {  // backward product of tile i (T in shared memory) into D2[i & 1]
        const int b = i & 1;
        if (!wait_bounded(tready(b), (uint32_t)((i >> 1) & 1), ab)) return false;
        if (!wait_bounded(d2empty(b), (uint32_t)(((i >> 1) & 1) ^ 1), ab)) return false;
        tc_fence_after();
        const uint32_t dacc = tmem + 256u + (uint32_t)(b * 128);
        for (int kt = 0; kt < KT; ++kt) {
          const unsigned long long td = dT + (uint32_t)(b * KT + kt) * (tkt >> 4);
          const int nk = min(4, (a.C - kt * kKTile + 15) >> 4);
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            if (kk < nk) {
              // K step kg: rows 16 kg.. of every W1 tile (two row groups of 1024 bytes each); the M atoms
              // (W1's K tiles) w1kt bytes apart; lo rows VR * 128 bytes after the hi rows
              const uint32_t ka = sW1 + 2048u * (uint32_t)(kt * 4 + kk);
              const unsigned long long wd = mn128_desc(ka, w1kt, 1024u);
              const unsigned long long wdl = mn128_desc(ka + (uint32_t)a.VR * 128u, w1kt, 1024u);
              tc_mma(dacc, wd, td + 2u * kk, idesc2, (kt > 0 || kk > 0) ? 1u : 0u);
              tc_mma(dacc, wd, td + tlo + 2u * kk, idesc2, 1u);
              tc_mma(dacc, wdl, td + 2u * kk, idesc2, 1u);
            }
          }
        }
        tc_commit(d2full(b));
        return true;
      };
      if (ok && nmine > 0) ok = stage1(0);
      for (int i = 0; ok && i < nmine; ++i) {
        if (i + 1 < nmine && !(ok = stage1(i + 1))) break;
        ok = stage2(i);
      }
      tc_commit(drain);  // every MMA this thread issued is complete once `drain` fires
      const unsigned long long t0 = gtimer();
      while (!mbar_try_wait(drain, 0) && gtimer() - t0 < kWaitLimitNs) {
      }
    }
    __syncwarp();
  } else if (warp >= 2) {
    // ---------------- epilogue: four warps per TMEM lane quadrant, warp h of a quadrant taking the 16-column
    // chunks h*16 + 64*j
    const int q = warp & 3, h = (warp - 2) >> 2;
    const int trow = q * 32 + lane;
    const int J1 = (a.Np - h * 16 + 63) / 64;  // stage-1 chunks of this warp (at most 2)
    // stage 1 of tile i: v = D1[row][c'] * G(row, c') * 2^-sG in FP32 (as the per-pass kernel), then
    // T[row][c'] = (bf16(v), bf16(v - hi)); rows past the grid hold zeros
    auto epi1 = [&](int i) {
      const int tile = (int)blockIdx.x + i * (int)gridDim.x;
      const int b = i & 1;
      const int r = tile * kTileRows + trow;
      const bool valid = r < a.rows;
      const int ia = valid ? r / a.B1 : 0;
      const int ib = valid ? r - ia * a.B1 : 0;
      const float sab = valid ? a.lamA[ia] + a.lamB[ib] : 0.0f;
      const bool null_row = a.singular && ia == 0 && ib == 0;
      if (!__all_sync(0xffffffffu, wait_bounded(d1full(b), (uint32_t)((i >> 1) & 1), ab))) return false;
      tc_fence_after();
      const uint32_t tacc = tmem + (uint32_t)(b * 128) + ((uint32_t)(q * 32) << 16);
      uint32_t t0[16], t1[16];
      if (J1 > 0) tc_ld16_issue(tacc + (uint32_t)(h * 16), t0);
      if (J1 > 1) tc_ld16_issue(tacc + (uint32_t)(h * 16 + 64), t1);
      if (J1 > 0) tc_ld16_wait(t0);
      if (J1 > 1) tc_ld16_wait(t1);
      tc_fence_before();
      mbar_arrive(d1empty(b));
      auto put = [&](int c0, const uint32_t (&t)[16]) {
        float v[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) v[k] = __uint_as_float(t[k]);
        const float4* lc4 = reinterpret_cast<const float4*>(a.lamC + c0);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const float4 l = __ldg(lc4 + k);
          v[4 * k + 0] *= rcp_approx(sab + l.x) * a.gscale;
          v[4 * k + 1] *= rcp_approx(sab + l.y) * a.gscale;
          v[4 * k + 2] *= rcp_approx(sab + l.z) * a.gscale;
          v[4 * k + 3] *= rcp_approx(sab + l.w) * a.gscale;
        }
        if (null_row && c0 == 0) v[0] = 0.0f;
        uint32_t ph[8], pl[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const __nv_bfloat162 h2 = __floats2bfloat162_rn(v[2 * k], v[2 * k + 1]);
          const float2 hf = __bfloat1622float2(h2);
          const __nv_bfloat162 l2 = __floats2bfloat162_rn(v[2 * k] - hf.x, v[2 * k + 1] - hf.y);
          ph[k] = valid ? *reinterpret_cast<const uint32_t*>(&h2) : 0u;
          pl[k] = valid ? *reinterpret_cast<const uint32_t*>(&l2) : 0u;
        }
        // 128-byte swizzle: 16-byte piece p of row trow sits at piece p ^ (trow % 8); lo one tile further
        const uint32_t rowa = sT + (uint32_t)(b * KT + (c0 >> 6)) * tkt + (uint32_t)trow * 128u;
        const uint32_t p0 = (uint32_t)((c0 & 63) >> 3);
#pragma unroll
        for (int k = 0; k < 2; ++k) {
          const uint32_t off = ((p0 + k) ^ (uint32_t)(trow & 7)) << 4;
          asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(rowa + off), "r"(ph[4 * k]),
                       "r"(ph[4 * k + 1]), "r"(ph[4 * k + 2]), "r"(ph[4 * k + 3])
                       : "memory");
          asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(rowa + (uint32_t)kTBytes + off),
                       "r"(pl[4 * k]), "r"(pl[4 * k + 1]), "r"(pl[4 * k + 2]), "r"(pl[4 * k + 3])
                       : "memory");
        }
      };
      if (J1 > 0) put(h * 16, t0);
      if (J1 > 1) put(h * 16 + 64, t1);
      // generic-proxy writes of T -> the tensor core's (async-proxy) reads
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_arrive(tready(b));
      return true;
    };
    // stage 2 of tile i: thread = output index c = q*32 + lane, chunk = 16 consecutive rows; the stores of
    // the per-pass kernel's form 2 (hi and lo planes)
    auto epi2 = [&](int i) {
      const int tile = (int)blockIdx.x + i * (int)gridDim.x;
      const int b = i & 1;
      const int row0 = tile * kTileRows;
      if (!__all_sync(0xffffffffu, wait_bounded(d2full(b), (uint32_t)((i >> 1) & 1), ab))) return false;
      tc_fence_after();
      const uint32_t tacc = tmem + 256u + (uint32_t)(b * 128) + ((uint32_t)(q * 32) << 16);
      uint32_t t0[16], t1[16];
      tc_ld16_issue(tacc + (uint32_t)(h * 16), t0);
      tc_ld16_issue(tacc + (uint32_t)(h * 16 + 64), t1);
      tc_ld16_wait(t0);
      tc_ld16_wait(t1);
      tc_fence_before();
      mbar_arrive(d2empty(b));
      const int c = q * 32 + lane;
      auto out = [&](int c0, const uint32_t (&t)[16]) {
        const int r0 = row0 + c0;
        if (r0 >= a.rows || c >= a.Cout) return;
        float v[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) v[k] = __uint_as_float(t[k]);
        int ia = r0 / a.B;
        int ib = r0 - ia * a.B;
        if (a.vec && ib + 16 <= a.B && r0 + 16 <= a.rows) {
          store16<Bf16Pair>(a.out, a.oplane, (long long)ia * a.oa + ib + (long long)c * a.oc, v);
        } else {
#pragma unroll
          for (int k = 0; k < 16; ++k) {
            if (r0 + k < a.rows)
              store_out<Bf16Pair>(a.out, a.oplane, (long long)ia * a.oa + (long long)ib * a.ob + (long long)c * a.oc,
                                  v[k]);
            if (++ib == a.B) {
              ib = 0;
              ++ia;
            }
          }
        }
      };
      out(h * 16, t0);
      out(h * 16 + 64, t1);
      return true;
    };
    // T buffer i & 1 was last read by stage 2 of tile i-2, drained (epi2) before epi1 writes tile i
    bool ok = true;
    for (int i = 0; ok && i < nmine; ++i) {
      ok = epi1(i);
      if (ok && i > 0) ok = epi2(i - 1);
    }
    if (ok && nmine > 0) epi2(nmine - 1);
  }

  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512u) : "memory");
  }
}

struct TcStage {
  CUtensorMap tmX;
  CUtensorMap tmW;
  CUtensorMap tmR;  // R~ (16-bit) for the last pass of a solve; a copy of tmX when unused
  CUtensorMap tmO;  // the pass's output for TMA stores (args.tstore); a copy of tmX when unused
  CUtensorMap tmW2; // fused pair: the backward pass's eigenbasis; a copy of tmW otherwise
  int form;
  int pair;  // 1: k_modeprod_pair runs this pass and the next one
  TcArgs args;
  void* out;  // output buffer of a pass that is not the last
  int grid;
  int ntiles;  // 128-row tiles of the pass (the persistent CTAs stride over them)
  size_t smem;
};

// CTAs of a pass: one per SM, or fewer so that each takes at least sweep_grain / 8 row tiles (plans
// solved many at once leave SMs to one another's launches).
int tc_grid(const tpcg_plan* p, int ntiles) {
  const int per = std::max(1, p->sweep_grain / 8);
  return std::max(1, std::min((ntiles + per - 1) / per, p->num_sms));
}

struct TcPlan {
  bool tf32 = false;  // TF32 form: FP32 containers, eigenbasis streamed, one launch per pass
  bool split = false;  // split BF16 form: hi/lo planes, three MMAs per K step, eigenbasis streamed, one launch
                       // per pass
  std::vector<TcStage> stages;  // one launch per pass of Algorithm 7
  std::vector<TcStage> fused;   // the same with the pass pair around G in one launch (empty when not possible)
  bool fp16 = false;
};

EncodeTiledFn encoder() { return tma_encoder(); }

// Rows of the 16-bit copy of R, 16 x 128 boxes with the 32-byte swizzle (last pass).
int encode_r(CUtensorMap* map, const void* gaddr, int inner, long long outer, long long pitch_elems, bool fp16) {
  EncodeTiledFn cuTensorMapEncodeTiled = encoder();
  if (!cuTensorMapEncodeTiled) return -1;
  cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)outer};
  cuuint64_t strides[1] = {(cuuint64_t)pitch_elems * 2};
  cuuint32_t box[2] = {16, (cuuint32_t)kTileRows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = cuTensorMapEncodeTiled(map, fp16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16,
                                      2, const_cast<void*>(gaddr), dims, strides,
                                      box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B,
                                      CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? 0 : -1;
}

// The output of a pass as boxes of 16 contiguous elements x 32 lanes (one epilogue warp's chunk).
// Form 1 (lane = row, contiguous output index): 2D {Cout, rows}, rows of one pitch.  Form 2 (lane =
// output index, contiguous rows): 3D {B, Cout, A} or, when A has the smaller stride, {B, A, Cout}.
// Returns -1 when the layout does not fit these maps (the pass then stores directly).
int encode_out(CUtensorMap* map, void* gaddr, int esize, bool fp16, int form, const TcArgs& a, int* tperm) {
  EncodeTiledFn cuTensorMapEncodeTiled = encoder();
  if (!cuTensorMapEncodeTiled) return -1;
  const CUtensorMapDataType dt = (esize == 4) ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                              : (fp16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16);
  const CUtensorMapSwizzle sw = (esize == 4) ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B;
  CUresult r;
  if (form == 1) {
    if (!(a.B == 1 || a.oa == (long long)a.B * a.ob)) return -1;
    const long long pitch = (a.B == 1) ? a.oa : a.ob;
    if (pitch <= 0 || (pitch * esize) % 16 != 0) return -1;
    cuuint64_t dims[2] = {(cuuint64_t)a.Cout, (cuuint64_t)a.rows};
    cuuint64_t strides[1] = {(cuuint64_t)(pitch * esize)};
    cuuint32_t box[2] = {16, 32};
    cuuint32_t estr[2] = {1, 1};
    r = cuTensorMapEncodeTiled(map, dt, 2, gaddr, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, sw,
                               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    *tperm = 0;
  } else {
    if (a.ob != 1 || a.B % 16 != 0 || (a.oc * esize) % 16 != 0 || (a.oa * esize) % 16 != 0) return -1;
    const int A = a.rows / a.B;
    const bool perm = a.oa < a.oc;
    cuuint64_t dims[3] = {(cuuint64_t)a.B, (cuuint64_t)(perm ? A : a.Cout), (cuuint64_t)(perm ? a.Cout : A)};
    cuuint64_t strides[2] = {(cuuint64_t)((perm ? a.oa : a.oc) * esize), (cuuint64_t)((perm ? a.oc : a.oa) * esize)};
    cuuint32_t box[3] = {16, perm ? 1u : 32u, perm ? 32u : 1u};
    cuuint32_t estr[3] = {1, 1, 1};
    r = cuTensorMapEncodeTiled(map, dt, 3, gaddr, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, sw,
                               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    *tperm = perm ? 1 : 0;
  }
  return r == CUDA_SUCCESS ? 0 : -1;
}

// Operands of the tensor core: FP16, BF16 or (TF32 form) FP32 containers.
enum class OpType { kF16, kBF16, kF32 };

int encode_2d(CUtensorMap* map, const void* gaddr, int inner, long long outer, int pitch_elems, int box_inner,
              int box_outer, OpType ty) {
  EncodeTiledFn cuTensorMapEncodeTiled = encoder();
  if (!cuTensorMapEncodeTiled) return -1;
  const int esz = (ty == OpType::kF32) ? 4 : 2;
  cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)outer};
  cuuint64_t strides[1] = {(cuuint64_t)pitch_elems * esz};
  cuuint32_t box[2] = {(cuuint32_t)box_inner, (cuuint32_t)box_outer};
  cuuint32_t estr[2] = {1, 1};
  const CUtensorMapDataType dt = ty == OpType::kF32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                 : (ty == OpType::kF16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16);
  CUresult r = cuTensorMapEncodeTiled(map, dt, 2, const_cast<void*>(gaddr), dims,
                                      strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                      CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? 0 : -1;
}

// A split-form operand: the BF16 hi plane and, plane_elems further, the lo plane, as one 3D map
// {inner, outer, 2} whose boxes {box_inner, box_outer, 2} land as the hi tile followed by the lo tile.
int encode_pair(CUtensorMap* map, const void* gaddr, int inner, long long outer, int pitch_elems, long long plane_elems,
                int box_inner, int box_outer) {
  EncodeTiledFn cuTensorMapEncodeTiled = encoder();
  if (!cuTensorMapEncodeTiled) return -1;
  if (plane_elems < outer * pitch_elems || (plane_elems * 2) % 16 != 0) return -1;
  cuuint64_t dims[3] = {(cuuint64_t)inner, (cuuint64_t)outer, 2};
  cuuint64_t strides[2] = {(cuuint64_t)pitch_elems * 2, (cuuint64_t)plane_elems * 2};
  cuuint32_t box[3] = {(cuuint32_t)box_inner, (cuuint32_t)box_outer, 2};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = cuTensorMapEncodeTiled(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(gaddr), dims, strides,
                                      box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                      CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? 0 : -1;
}

template <int FORM, class InT, class OutT, bool FINAL>
int set_smem_attr(size_t smem) {
  return cudaFuncSetAttribute(k_modeprod_tc<FORM, InT, OutT, FINAL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)smem) == cudaSuccess
             ? 0
             : -1;
}

template <class InT>
int set_all_smem_attrs() {
  int bad = 0;
  bad |= set_smem_attr<1, InT, InT, false>(kMaxSmem);
  bad |= set_smem_attr<2, InT, InT, false>(kMaxSmem);
  bad |= set_smem_attr<1, InT, float, false>(kMaxSmem);
  bad |= set_smem_attr<1, InT, float, true>(kMaxSmem);
  bad |= cudaFuncSetAttribute(k_modeprod_pair<InT>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem) ==
                 cudaSuccess
             ? 0
             : -1;
  return bad;
}

int set_tf32_smem_attrs() {
  int bad = 0;
  bad |= set_smem_attr<1, float, float, false>(kMaxSmem);
  bad |= set_smem_attr<2, float, float, false>(kMaxSmem);
  bad |= set_smem_attr<1, float, float, true>(kMaxSmem);
  return bad;
}

int set_split_smem_attrs() {
  int bad = 0;
  bad |= set_smem_attr<1, Bf16Pair, Bf16Pair, false>(kMaxSmem);
  bad |= set_smem_attr<2, Bf16Pair, Bf16Pair, false>(kMaxSmem);
  bad |= set_smem_attr<1, Bf16Pair, float, false>(kMaxSmem);
  bad |= set_smem_attr<1, Bf16Pair, float, true>(kMaxSmem);
  if (cudaFuncSetAttribute(k_modeprod_pair_split, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem) !=
      cudaSuccess)
    bad |= -1;
  return bad;
}

template <int FORM, class InT, class OutT, bool FINAL>
void launch(const TcStage& s, const TcArgs& a, cudaStream_t stream) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)s.grid);
  cfg.blockDim = dim3(TcWarps<FINAL>::threads);
  cfg.dynamicSmemBytes = s.smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;  // see griddepcontrol in the kernel
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, k_modeprod_tc<FORM, InT, OutT, FINAL>, s.tmX, s.tmW, s.tmR, s.tmO, a);
}

template <class InT>
void launch_pair(const TcStage& s, const TcArgs& a, cudaStream_t stream) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)s.grid);
  cfg.blockDim = dim3(kPairThreads);
  cfg.dynamicSmemBytes = s.smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, k_modeprod_pair<InT>, s.tmX, s.tmW, s.tmW2, s.tmO, a);
}

void launch_pair_split(const TcStage& s, const TcArgs& a, cudaStream_t stream) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)s.grid);
  cfg.blockDim = dim3(kPairSplitThreads);
  cfg.dynamicSmemBytes = s.smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, k_modeprod_pair_split, s.tmX, s.tmW, s.tmW2, a);
}

template <class InT>
void launch_stage(const TcStage& s, const TcArgs& a, bool last, bool final_pcg, cudaStream_t stream) {
  if (s.pair) {
    // (no fused pair in the TF32 form; the split form has a kernel of its own)
    if constexpr (KShape<InT>::split) launch_pair_split(s, a, stream);
    else if constexpr (!KShape<InT>::tf32) launch_pair<InT>(s, a, stream);
  } else if (!last) {
    if (s.form == 1) launch<1, InT, InT, false>(s, a, stream);
    else launch<2, InT, InT, false>(s, a, stream);
  } else if (final_pcg) {
    launch<1, InT, float, true>(s, a, stream);
  } else {
    launch<1, InT, float, false>(s, a, stream);
  }
}

// Smallest positive eigenvalue sum: the largest entry of G.
double smallest_positive_sum(const tpcg_plan* p) {
  std::vector<double> cand[3];
  for (int m = 0; m < 3; ++m) {
    std::vector<double> l = p->ax[m].lam;
    std::sort(l.begin(), l.end());
    l.erase(std::unique(l.begin(), l.end()), l.end());
    cand[m].assign(l.begin(), l.begin() + std::min<size_t>(2, l.size()));
  }
  double best = 0.0;
  for (double x : cand[0])
    for (double y : cand[1])
      for (double z : cand[2]) {
        const double v = x + y + z;
        if (v > 1e-300 && (best == 0.0 || v < best)) best = v;
      }
  return best;
}

}  // namespace

// FP16 range: R enters at unit RMS, so intermediates of the forward products are bounded by sqrt(N);
// after G they are bounded by sqrt(N) * max G, which 2^-sG brings under 2^14 (below the FP16 maximum
// 65504).
int tc_fp16_g_exponent(const tpcg_plan* p) {
  const double smin = smallest_positive_sum(p);
  const double bound = std::sqrt((double)p->N) / (smin > 0 ? smin : 1.0);
  return std::max(0, (int)std::ceil(std::log2(bound / 16384.0)));
}

bool slab_applicable(const tpcg_plan* p);
int slab_plan_setup(tpcg_plan* p);
void slab_plan_release(tpcg_plan* p);
int slab_launches_per_apply(const tpcg_plan* p);
int run_precond_slab(const tpcg_plan* p, float* Z, SolveState* st);

int tc_plan_setup(tpcg_plan* p) {
  if (p->prec != TPCG_MIXED_BF16 && p->prec != TPCG_MIXED_FP16 && p->prec != TPCG_MIXED_TF32 &&
      p->prec != TPCG_MIXED_BF16X3)
    return TPCG_ERR_UNSUPPORTED;
  TcPlan* tp = new TcPlan();
  tp->fp16 = (p->prec == TPCG_MIXED_FP16);
  tp->tf32 = (p->prec == TPCG_MIXED_TF32);
  tp->split = (p->prec == TPCG_MIXED_BF16X3);
  const OpType oty = tp->tf32 ? OpType::kF32 : (tp->fp16 ? OpType::kF16 : OpType::kBF16);
  const int ktile = tp->tf32 ? 32 : kKTile;  // elements per 128-byte K tile
  // FP16 range: R enters at unit RMS, so intermediates of the forward passes
  // are bounded by sqrt(N); after G they are bounded by sqrt(N) * max G,
  // which 2^-sG brings under 2^14 (below the FP16 maximum 65504).
  const int sG = tp->fp16 ? tc_fp16_g_exponent(p) : 0;
  const int ns = (int)p->stages.size();
  // Launch parameters of pass si reading xin and writing out_addr (the plan's Z for the last pass).
  auto build_one = [&](int si, const void* xin, void* out_addr, TcStage& st) -> int {
    const StageParams& sp = p->stages[si];
    st = TcStage{};
    // form 1 (thread = row) when the output index is contiguous, form 2 (thread = output index)
    // when consecutive rows are: either way a thread owns 16 contiguous outputs
    st.form = (sp.oc == 1) ? 1 : 2;
    TcArgs& a = st.args;
    a.C = sp.C;
    a.KT = (sp.C + ktile - 1) / ktile;
    a.Cout = sp.Cout;
    a.Np = ((sp.Cout + 15) / 16) * 16;
    a.MB = (sp.Cout + 127) / 128;
    a.VR = (st.form == 1) ? ((sp.Cout + 7) / 8) * 8 : a.MB * 128;
    if (st.form == 1) a.VR = std::max(a.VR, a.Np);
    a.acc_cols = (st.form == 1) ? a.Np : a.MB * 128;
    int cols = 32;
    while (cols < 2 * a.acc_cols) cols <<= 1;
    a.tmem_cols = cols;
    a.rows = sp.A * sp.B;
    a.B = sp.B;
    a.B1 = sp.B;
    a.oa = sp.oa;
    a.ob = sp.ob;
    a.oc = sp.oc;
    a.scale = sp.scale;
    if (st.form == 2 && (sp.scale || sp.final_stage)) return TPCG_ERR_UNSUPPORTED;  // form-1 epilogues only
    if (st.form == 1)
      a.vec = (sp.final_stage ? (sp.oa % 4 == 0 && sp.ob % 4 == 0) : (sp.oa % 8 == 0 && sp.ob % 8 == 0)) ? 1 : 0;
    else
      a.vec = (sp.ob == 1 && sp.oa % 8 == 0 && sp.oc % 8 == 0 && sp.B % 8 == 0) ? 1 : 0;
    a.singular = p->singular ? 1 : 0;
    a.lamA = p->d_lam32[sp.lamA];
    a.lamB = p->d_lam32[sp.lamB];
    a.lamC = p->d_lam32[sp.lamC];
    a.N = p->N;
    a.err = p->d_err;
    a.last = sp.final_stage;
    a.sG = sG;
    a.gscale = std::ldexp(1.0f, -sG);
    // FP16 and split: R~ holds R * 2^shift (the FP16 range, and the split's lo words far from BF16's
    // underflow); the last pass undoes the scale on Z
    a.shift_src = (tp->fp16 || tp->split) ? &p->d_state->lp_shift_applied : nullptr;
    // TF32 and split: the eigenbasis (up to 256 x 256 FP32 or BF16 pairs, 256 KB) does not fit next to the
    // stages; each stage then carries its K tile of the eigenbasis with the data tile (split: the hi and lo
    // tiles of both).  (Keeping 128 eigenbasis rows resident per CTA, two CTAs per tile, measured slower:
    // the ring left beside them is too shallow to hide the loads' latency behind the epilogue's stores.)
    a.wstream = (tp->tf32 || tp->split) ? 1 : 0;
    a.sbytes = (tp->split ? 2 : 1) * (kStageBytes + (a.wstream ? a.VR * 128 : 0));
    const size_t sbytes = (size_t)a.sbytes;
    const size_t vbytes = a.wstream ? 0 : (size_t)a.KT * a.VR * 128;
    size_t fixed = 1024 + vbytes + 512;  // alignment, eigenbasis, barriers and the TMEM address
    if (a.tmem_cols > 512 || a.VR > 256 || fixed + 2 * sbytes > (size_t)kMaxSmem) return TPCG_ERR_UNSUPPORTED;
    // outputs by TMA stores through per-warp staging when the layout allows
    const bool last = sp.final_stage != 0;
    const int esz = (last || tp->tf32) ? 4 : 2;
    st.out = out_addr;
    st.tmO = st.tmX;
    // (the split form stores its two planes directly)
    a.tstore = (!tp->split && encode_out(&st.tmO, out_addr, esz, tp->fp16, st.form, a, &a.tperm) == 0) ? 1 : 0;
    a.oplane = (long long)p->t_plane;
    a.rplane = (long long)p->lp_plane;
    // staging bytes: two [32][16] boxes per epilogue warp (sixteen warps; eight in the last pass of a solve)
    const size_t stage_plain = a.tstore ? (size_t)TcWarps<false>::epi * 2 * 32 * 16 * esz : 0;
    const size_t stage_final = (a.tstore && last) ? (size_t)TcWarps<true>::epi * 2 * 32 * 16 * esz : 0;
    // last pass of a solve: R~ (the first pass's input, rows of pitch pitch16[0], a multiple of 8
    // elements) by TMA through the largest ring (up to kRHalf slots per half) that leaves two stages
    a.rpitch = p->pitch16[0];
    a.rhalf = 0;
    if (last && st.form == 1 && !tp->tf32 && !tp->split) {  // (TF32 and split read R~ with global loads)
      const size_t room = (size_t)kMaxSmem - fixed - 2 * sbytes;
      const size_t rh = room > stage_final ? (room - stage_final) / (2 * (size_t)kRBytes) : 0;
      a.rhalf = (int)std::min<size_t>(kRHalf, rh);
    }
    a.rtma = (a.rhalf >= 2) ? 1 : 0;
    if (!a.rtma) a.rhalf = 0;
    a.aux = (int)std::max(stage_plain, (size_t)(2 * a.rhalf * kRBytes) + stage_final);
    if (fixed + (size_t)a.aux + 2 * sbytes > (size_t)kMaxSmem) {  // no room for staging: direct stores
      a.tstore = 0;
      a.aux = 2 * a.rhalf * kRBytes;
    }
    fixed += (size_t)a.aux;
    a.NS = (int)std::min<size_t>(8, (kMaxSmem - fixed) / sbytes);
    st.smem = fixed + (size_t)a.NS * sbytes;
    const int ntiles = (a.rows + kTileRows - 1) / kTileRows;
    st.ntiles = ntiles;
    st.grid = tc_grid(p, ntiles);
    const int wpitch = p->pitch16[sp.axis];
    if (tp->split) {
      const long long xplane = (long long)((xin == p->d_Rlp) ? p->lp_plane : p->t_plane);
      if (encode_pair(&st.tmX, xin, sp.C, (long long)a.rows, sp.in_pitch, xplane, ktile, kTileRows) ||
          encode_pair(&st.tmW, p->d_Wt16[sp.axis][sp.dir], sp.C, sp.Cout, wpitch, (long long)sp.Cout * wpitch, ktile,
                      a.VR))
        return TPCG_ERR_CUDA;
    } else if (encode_2d(&st.tmX, xin, sp.C, (long long)a.rows, sp.in_pitch, ktile, kTileRows, oty) ||
               encode_2d(&st.tmW, p->d_Wt16[sp.axis][sp.dir], sp.C, sp.Cout, wpitch, ktile, a.VR, oty))
      return TPCG_ERR_CUDA;
    st.tmW2 = st.tmW;
    st.tmR = st.tmX;
    if (a.rtma && encode_r(&st.tmR, p->d_Rlp, sp.Cout, (long long)a.rows, a.rpitch, tp->fp16)) return TPCG_ERR_CUDA;
    return TPCG_OK;
  };
  // Passes si (forward, with G, form 1) and si + 1 (backward along the same axis, form 2) as one
  // k_modeprod_pair launch; TPCG_ERR_UNSUPPORTED when the pair does not fit its layout rules.
  auto build_pair = [&](int si, const void* xin, void* out_addr, TcStage& st) -> int {
    if (si + 1 >= ns || tp->tf32) return TPCG_ERR_UNSUPPORTED;
    const StageParams& s1 = p->stages[si];
    const StageParams& s2 = p->stages[si + 1];
    const bool shape_ok = s1.scale && !s1.final_stage && s1.oc == 1 && !s2.final_stage && s2.oc != 1 &&
                          s1.axis == s2.axis && s1.dir != s2.dir && s1.C == s1.Cout && s2.C == s1.C &&
                          s2.Cout == s1.C && s1.C % 16 == 0 && s1.C <= 128 && s1.A * s1.B == s2.A * s2.B &&
                          (s1.B == 1 || s1.oa == (long long)s1.B * s1.ob) &&
                          ((s1.B == 1) ? s1.oa : s1.ob) == (long long)s2.in_pitch;  // row r of s1's output = row r of s2's input
    if (!shape_ok) return TPCG_ERR_UNSUPPORTED;
    TcStage f{}, b{};
    int rc;
    if ((rc = build_one(si, xin, out_addr, f)) || (rc = build_one(si + 1, xin, out_addr, b))) return rc;
    if (tp->split) {  // k_modeprod_pair_split: both split eigenbases resident, one T buffer, direct stores
      if (f.form != 1 || b.form != 2 || b.args.MB != 1) return TPCG_ERR_UNSUPPORTED;
      st = b;
      st.pair = 1;
      st.tmX = f.tmX;   // the forward pass's input pair, boxes {64, 128, 2}
      st.tmW = f.tmW;   // W1: the forward eigenbasis pair, boxes {64, VR, 2}
      st.tmW2 = b.tmW;  // (unused: stage 2 reads W1 transposed)
      TcArgs& a = st.args;
      a.Np = f.args.Np;
      a.VR = f.args.VR;
      a.B1 = s1.B;
      a.scale = 1;
      a.gscale = f.args.gscale;
      a.lamA = f.args.lamA;
      a.lamB = f.args.lamB;
      a.lamC = f.args.lamC;
      // alignment, the forward eigenbasis (hi and lo; stage 2 reads it transposed), two T buffers (hi and
      // lo), barriers and the TMEM address
      const size_t fixed = 1024 + (size_t)a.KT * 2 * a.VR * 128 + 2 * (size_t)a.KT * 2 * kTBytes + 512;
      if (fixed + 2 * (size_t)kStageBytes > (size_t)kMaxSmem) return TPCG_ERR_UNSUPPORTED;
      a.NS = (int)std::min<size_t>(8, (kMaxSmem - fixed) / (2 * (size_t)kStageBytes));
      st.smem = fixed + (size_t)a.NS * 2 * kStageBytes;
      return TPCG_OK;
    }
    if (f.form != 1 || b.form != 2 || !b.args.tstore || b.args.MB != 1 || b.args.B % 16 != 0)
      return TPCG_ERR_UNSUPPORTED;
    st = b;
    st.pair = 1;
    st.tmX = f.tmX;
    st.tmW = f.tmW;  // W1: the forward eigenbasis, rows padded to a multiple of 8
    if (encode_2d(&st.tmW2, p->d_Wt16[s2.axis][s2.dir], s2.C, s2.Cout, p->pitch16[s2.axis], kKTile, 128, oty))
      return TPCG_ERR_CUDA;
    TcArgs& a = st.args;
    a.Np = f.args.Np;
    a.VR = f.args.VR;
    a.B1 = s1.B;
    a.scale = 1;
    a.lamA = f.args.lamA;
    a.lamB = f.args.lamB;
    a.lamC = f.args.lamC;
    // alignment, both eigenbases, the two T buffers, the output staging (two FP16/BF16 [32][16] boxes per
    // epilogue warp), barriers and the TMEM address
    const size_t fixed = 1024 + (size_t)a.KT * (a.VR + 128) * 128 + 2 * (size_t)a.KT * kTBytes +
                         (size_t)kPairEpi * 2 * 32 * 16 * 2 + 512;
    if (fixed + 2 * (size_t)kStageBytes > (size_t)kMaxSmem) return TPCG_ERR_UNSUPPORTED;
    a.NS = (int)std::min<size_t>(8, (kMaxSmem - fixed) / kStageBytes);
    st.smem = fixed + (size_t)a.NS * kStageBytes;
    return TPCG_OK;
  };
  const int bad = tp->tf32    ? set_tf32_smem_attrs()
                  : tp->split ? set_split_smem_attrs()
                              : (tp->fp16 ? set_all_smem_attrs<__half>() : set_all_smem_attrs<__nv_bfloat16>());
  if (bad) {
    delete tp;
    return TPCG_ERR_CUDA;
  }
  int rc = TPCG_OK;
  for (int si = 0; si < ns && rc == TPCG_OK; ++si) {
    TcStage st{};
    const bool last = (si == ns - 1);
    rc = build_one(si, (si == 0) ? p->d_Rlp : p->d_T[(si - 1) & 1], last ? p->d_Z : p->d_T[si & 1], st);
    if (rc == TPCG_OK) tp->stages.push_back(st);
  }
  // the fused launch sequence: launch li reads the previous launch's output and writes d_T[li % 2]
  int sf = -1;
  for (int si = 0; si + 1 < ns && sf < 0; ++si)
    if (p->stages[si].scale) sf = si;
  if (rc == TPCG_OK && sf >= 0) {
    const void* prev = p->d_Rlp;
    for (int si = 0, li = 0; si < ns; ++li) {
      const bool pair = (si == sf);
      const bool last = (si + (pair ? 1 : 0) == ns - 1);
      void* outp = last ? p->d_Z : p->d_T[li & 1];
      TcStage st{};
      const int r = pair ? build_pair(si, prev, outp, st) : build_one(si, prev, outp, st);
      if (r != TPCG_OK) {  // the pair does not fit here: keep the one-launch-per-pass sequence only
        tp->fused.clear();
        break;
      }
      tp->fused.push_back(st);
      prev = outp;
      si += pair ? 2 : 1;
    }
  }
  if (rc != TPCG_OK) {
    delete tp;
    return rc;
  }
  p->tc_state = tp;
  if (slab_applicable(p)) {
    const int r = slab_plan_setup(p);
    if (r != TPCG_OK && r != TPCG_ERR_UNSUPPORTED) return r;
  }
  return TPCG_OK;
}

// Re-derive the CTA counts after the plan's sweep grain changed.
void tc_apply_grain(tpcg_plan* p) {
  TcPlan* tp = reinterpret_cast<TcPlan*>(p->tc_state);
  if (!tp) return;
  for (auto* v : {&tp->stages, &tp->fused})
    for (TcStage& st : *v) st.grid = tc_grid(p, st.ntiles);
}

int tc_launches_per_apply(const tpcg_plan* p) {
  const TcPlan* tp = reinterpret_cast<const TcPlan*>(p->tc_state);
  if (!tp) return 0;
  if (p->tc_slab && p->slab_state) return slab_launches_per_apply(p);
  return (int)((p->tc_fuse && !tp->fused.empty()) ? tp->fused.size() : tp->stages.size());
}

void tc_plan_release(tpcg_plan* p) {
  slab_plan_release(p);
  delete reinterpret_cast<TcPlan*>(p->tc_state);
  p->tc_state = nullptr;
}

// R (already converted to BF16 in d_Rlp) -> Z (FP32).  With st != nullptr the
// last pass performs the PCG finalize.
int run_precond_tc(const tpcg_plan* p, float* Z, SolveState* st) {
  const TcPlan* tp = reinterpret_cast<const TcPlan*>(p->tc_state);
  if (!tp) return TPCG_ERR_UNSUPPORTED;
  if (p->tc_slab && p->slab_state && (void*)Z == p->d_Z) return run_precond_slab(p, Z, st);
  const std::vector<TcStage>& seq = (p->tc_fuse && !tp->fused.empty()) ? tp->fused : tp->stages;
  const int ns = (int)seq.size();
  for (int si = 0; si < ns; ++si) {
    const TcStage& s = seq[si];
    TcArgs a = s.args;
    const bool last = (si == ns - 1);
    a.out = last ? (void*)Z : s.out;
    if (last && (void*)Z != p->d_Z) a.tstore = 0;  // the output map names the plan's Z buffer
    a.st = st;
    a.Rt = reinterpret_cast<const uint16_t*>(p->d_Rlp);
    a.partials = p->d_partials;
    LaunchScope ls(p, kKModeTC);
    if (tp->tf32) launch_stage<float>(s, a, last, st != nullptr, p->stream);
    else if (tp->split) launch_stage<Bf16Pair>(s, a, last, st != nullptr, p->stream);
    else if (tp->fp16) launch_stage<__half>(s, a, last, st != nullptr, p->stream);
    else launch_stage<__nv_bfloat16>(s, a, last, st != nullptr, p->stream);
  }
  return TPCG_OK;
}

}  // namespace tpcg
