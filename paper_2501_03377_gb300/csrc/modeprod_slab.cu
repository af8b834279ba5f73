// Frontal-slice form of the tensor-core preconditioner (Algorithm 7, Sec. 4.3.3).
//
// The six mode products of one application are grouped by where their data
// live.  The x and y products of Algorithm 7 act inside one frontal slice
// (a z-plane, q x n), the z products along the mode-3 fibres (tubes):
//   k_frontal_pair<fwd>   per z-plane t:  F1_t = V_y^T (V_x^T R~_t^T)^T   (x, then y)
//   k_tube_pair           per column block of the [t][q'][n'] array:
//                         F2 = V_z (G o (V_z^T F1))   (z forward, Hadamard step, z backward)
//   k_frontal_pair<bwd>   per z-plane t:  Z_t = V_y (V_x F2_t^T)^T   (x, then y) -> FP32 Z,
//                         with rho = <R~, Z>, sum Z and max |Z| in the last launch of a solve.
// Three launches and two intermediates per application (four launches when
// the z axis exceeds 128 points: the tube products then run as two
// launches).  Every launch chains two GEMMs through shared memory:
//   frontal step 1: D1[n'][q] = sum_n W1[n'][n] X[q][n]      (A = eigenbasis, B = the slice, K-major)
//           step 2: D2[q'][n'] = sum_q W2[q'][q] T[n'][q]    (T = round(D1), K-major in shared memory)
//   tube    stage 1: D1[t'][c] = sum_t W1[t'][t] F[t][c]    (B MN-major: the column index is contiguous)
//           stage 2: D2[t][c]  = sum_t' W2[t][t'] T[t'][c] (T = round(G o D1), MN-major in shared memory)
// so no pass permutes its output and every global access is a contiguous
// TMA box.  Intermediates are FP16 (scaled as in the per-pass kernels) or
// BF16 with FP32 accumulation in TMEM.
//
// Warps: 0 TMA producer, 1 MMA issuer (one thread), 2..17 epilogue (four per
// TMEM lane quadrant).  Every mbarrier wait is bounded (2 s); on expiry the
// CTA sets the plan's error word, drains what it issued and frees TMEM.
#include <algorithm>
#include <cmath>
#include <vector>

#include "tc_ptx.cuh"

namespace tpcg {

namespace {
using namespace tcx;

constexpr int kSlabEpi = 16;
constexpr int kSlabThreads = (2 + kSlabEpi) * 32;       // tube pair: producer, MMA, epilogue
constexpr int kFrontalThreads = (3 + kSlabEpi) * 32;    // frontal pair: + the producer of the step-2 ring
constexpr int kFrontalRing2Warp = 2 + kSlabEpi;
constexpr int kBlk = 16384;  // one 128-row x 64-element K tile of a K-major operand (128-byte rows)
constexpr int kTubeCols = 128;  // columns of one tube tile (two MN-major atoms of 64)

struct SlabArgs {
  int n, q, t;             // grid nx, ny, nz
  // frontal pair
  int MB1, N1, KT1;        // step 1: 128-row blocks of n', N = q padded to 16, K tiles (64) of n
  int MB2, N2, KT2;        // step 2: 128-row blocks of q', N = n padded to 16, K tiles of q
  int NS1, NS2;            // ring stages
  uint32_t reg1;           // bytes of the step-1 ring (the slice-T overlays it)
  int stg;                 // output staging boxes per epilogue warp (1 or 2)
  // tube pair
  int MBz, KTz;            // 128-row blocks / K tiles (64) of the z axis
  int KS, KTs;             // K rows of one tube stage (64 or 128) and stages per column tile
  int ntiles;              // column tiles of q*n
  int NS;                  // ring stages
  int apply_g;             // single tube pass: multiply by G (forward) or not (backward)
  // common
  int last;                // output is Z (FP32): multiply by 2^(sG - s_R)
  int sG;
  float gscale;            // 2^-sG
  const int* shift_src;    // exponent the FP16 copy of R was scaled with (device), or null
  const float* lamx;
  const float* lamy;
  const float* lamz;
  int singular;
  const uint16_t* Rt;      // R~, the copy of R the first launch read (rows of rpitch elements)
  int rpitch;
  SolveState* st;
  double* partials;
  long long N;
  int* err;
};

// One [32][16] output box of an epilogue warp: staged in shared memory (swizzled rows) and written by a
// TMA store; with two staging buffers the store of one box overlaps the staging of the next.
template <class OutT>
struct BoxEmitter {
  uint32_t sOw;
  int nbuf;
  int cnt = 0;
  static constexpr uint32_t kBytes = 32u * 16u * (uint32_t)sizeof(OutT);
  __device__ __forceinline__ uint32_t stage(const float (&v)[16], int lane) {
    const uint32_t buf = sOw + (uint32_t)(nbuf == 2 ? (cnt & 1) : 0) * kBytes;
    if (cnt >= nbuf) {
      if (lane == 0) {
        if (nbuf == 2) asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
        else asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
      }
      __syncwarp();
    }
    stage_row<OutT>(buf, lane, v);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic writes -> async-proxy reads
    __syncwarp();
    ++cnt;
    return buf;
  }
  __device__ __forceinline__ void put3(const CUtensorMap* map, const float (&v)[16], int lane, int x0, int x1, int x2) {
    const uint32_t buf = stage(v, lane);
    if (lane == 0) {
      tma_store_3d(map, buf, x0, x1, x2);
      asm volatile("cp.async.bulk.commit_group;" ::: "memory");
    }
  }
  __device__ __forceinline__ void put2(const CUtensorMap* map, const float (&v)[16], int lane, int x0, int x1) {
    const uint32_t buf = stage(v, lane);
    if (lane == 0) {
      tma_store_2d(map, buf, x0, x1);
      asm volatile("cp.async.bulk.commit_group;" ::: "memory");
    }
  }
};

// Eight packed 16-bit values (FP16 or BF16, round to nearest even) of 16 FP32 values.
template <class T>
__device__ __forceinline__ void pack16(const float (&v)[16], uint32_t (&pk)[8]) {
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    if constexpr (std::is_same<T, __half>::value) {
      __half2 h2 = __floats2half2_rn(v[2 * k], v[2 * k + 1]);
      pk[k] = *reinterpret_cast<uint32_t*>(&h2);
    } else {
      __nv_bfloat162 h2 = __floats2bfloat162_rn(v[2 * k], v[2 * k + 1]);
      pk[k] = *reinterpret_cast<uint32_t*>(&h2);
    }
  }
}

// ------------------------------------------------------------------ frontal pair
// One CTA per z-plane (persistent over planes).  Step 1 streams the slice and
// the step-1 eigenbasis in 64-wide K tiles through a ring; the rounded D1
// (the slice after the x product, transposed) is written into shared memory
// over that ring as the K-major B operand of step 2, whose eigenbasis streams
// through a second ring.  TMEM: D1 blocks at columns b*N1, D2 blocks at b*N2
// (D2 is written once D1 has been drained).
template <class InT, class OutT, bool FINAL>
__global__ void __launch_bounds__(kFrontalThreads, 1)
    k_frontal_pair(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmA1,
                   const __grid_constant__ CUtensorMap tmA2, const __grid_constant__ CUtensorMap tmO, SlabArgs a) {
  if (a.st && a.st->done) return;
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t* sm = smem_raw + (base - raw);
  const int MB1 = a.MB1, MB2 = a.MB2, NS1 = a.NS1, NS2 = a.NS2;
  const uint32_t stage1 = (uint32_t)MB1 * kBlk + (uint32_t)a.N1 * 128u;  // eigenbasis K tile + slice K tile
  const uint32_t sR1 = base;                       // step-1 ring; the slice-T overlays it
  const uint32_t sT = base;
  const uint32_t sR2 = base + a.reg1;              // step-2 ring (one 128-row block per stage)
  const uint32_t sO = sR2 + (uint32_t)NS2 * kBlk;  // output staging
  constexpr uint32_t kOB = 32u * 16u * (uint32_t)sizeof(OutT);
  uint8_t* barp = sm + (sO - base) + (size_t)kSlabEpi * a.stg * kOB;
  const uint32_t bars = smem_u32(barp);
  auto full1 = [&](int s) { return bars + 8u * s; };
  auto empty1 = [&](int s) { return bars + 8u * (NS1 + s); };
  auto full2 = [&](int s) { return bars + 8u * (2 * NS1 + s); };
  auto empty2 = [&](int s) { return bars + 8u * (2 * NS1 + NS2 + s); };
  const uint32_t b0 = bars + 8u * (2 * NS1 + 2 * NS2);
  const uint32_t d1full = b0, tready = b0 + 8, d2full0 = b0 + 16, d2empty = b0 + 32, tfree = b0 + 40,
                 drain = b0 + 48;
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(barp + 8 * (2 * NS1 + 2 * NS2 + 7));
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_holder + 1);
  const Abort ab{abort_flag, a.err, a.st};

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < NS1; ++s) {
      mbar_init(full1(s), 1);
      mbar_init(empty1(s), 1);
    }
    for (int s = 0; s < NS2; ++s) {
      mbar_init(full2(s), 1);
      mbar_init(empty2(s), 1);
    }
    mbar_init(d1full, 1);
    mbar_init(tready, kSlabEpi * 32);
    mbar_init(d2full0, 1);
    mbar_init(d2full0 + 8, 1);
    mbar_init(d2empty, kSlabEpi * 32);
    mbar_init(tfree, 1);
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
  const int nplanes = a.t;
  const int nmine = nplanes > (int)blockIdx.x ? (nplanes - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;

  Acc32 red0, red1;
  float zmax = 0.0f;
  const int shR = (FINAL && a.st) ? a.st->lp_shift_applied : 0;
  const float rs = std::is_same<InT, __half>::value ? 1.0f : ldexpf(1.0f, shR);

  if (warp == 0) {
    // ---------------- TMA producer of the step-1 ring: lane 0 waits for a free stage, then lanes 0 and 1
    // issue the stage's two boxes (eigenbasis K tile, slice K tile) with one instruction
    asm volatile("griddepcontrol.wait;" ::: "memory");  // the slices are the previous launch's output
    int it1 = 0;
    bool ok = true;
    for (int i = 0; ok && i < nmine; ++i) {
      const int p = (int)blockIdx.x + i * (int)gridDim.x;
      // the slice-T of the previous plane overlays the step-1 ring: wait until step 2 has read it
      if (i > 0) {
        bool w = true;
        if (lane == 0) w = wait_bounded(tfree, (uint32_t)((i - 1) & 1), ab);
        if (!(ok = __shfl_sync(0xffffffffu, w, 0))) break;
      }
      for (int kt = 0; kt < a.KT1; ++kt, ++it1) {
        const int s = it1 % NS1;
        bool w = true;
        if (lane == 0) {
          w = wait_bounded(empty1(s), (uint32_t)(((it1 / NS1) & 1) ^ 1), ab);
          if (w) mbar_expect_tx(full1(s), stage1);
        }
        if (!(ok = __shfl_sync(0xffffffffu, w, 0))) break;
        const uint32_t st = sR1 + (uint32_t)s * stage1;
        if (lane < 2)
          tma_load_3d(lane ? st + (uint32_t)MB1 * kBlk : st, lane ? &tmX : &tmA1, kt * 64, 0, lane ? p : 0,
                      full1(s));
      }
    }
    if (!ok && lane == 0) {  // every issued load completes before the CTA may exit
      for (int j = (it1 > NS1 ? it1 - NS1 : 0); j < it1; ++j) {
        const unsigned long long t0 = gtimer();
        while (!mbar_try_wait(full1(j % NS1), (uint32_t)((j / NS1) & 1)) && gtimer() - t0 < kWaitLimitNs) {
        }
      }
    }
    __syncwarp();
  } else if (warp == kFrontalRing2Warp) {
    // ---------------- TMA producer of the step-2 ring (the eigenbasis of step 2, one 128-row block per
    // stage), running ahead of the step-1 producer
    if (lane == 0) {
      int it2 = 0;
      bool ok = true;
      for (int i = 0; ok && i < nmine; ++i)
        for (int b = 0; ok && b < MB2; ++b)
          for (int kt = 0; ok && kt < a.KT2; ++kt, ++it2) {
            const int s = it2 % NS2;
            if (!(ok = wait_bounded(empty2(s), (uint32_t)(((it2 / NS2) & 1) ^ 1), ab))) break;
            mbar_expect_tx(full2(s), kBlk);
            tma_load_2d(sR2 + (uint32_t)s * kBlk, &tmA2, kt * 64, b * 128, full2(s));
          }
      if (!ok) {
        for (int j = (it2 > NS2 ? it2 - NS2 : 0); j < it2; ++j) {
          const unsigned long long t0 = gtimer();
          while (!mbar_try_wait(full2(j % NS2), (uint32_t)((j / NS2) & 1)) && gtimer() - t0 < kWaitLimitNs) {
          }
        }
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issuer
      constexpr uint32_t fmt = std::is_same<InT, __half>::value ? 0u : 1u;
      const uint32_t idesc1 = idesc_f16kind(128, a.N1, fmt), idesc2 = idesc_f16kind(128, a.N2, fmt);
      int it1 = 0, it2 = 0;
      bool ok = true;
      for (int i = 0; ok && i < nmine; ++i) {
        if (i > 0 && !(ok = wait_bounded(d2empty, (uint32_t)((i - 1) & 1), ab))) break;
        tc_fence_after();
        // step 1: D1[b] = W1 block b . X^T over the K tiles of n
        for (int kt = 0; ok && kt < a.KT1; ++kt, ++it1) {
          const int s = it1 % NS1;
          if (!(ok = wait_bounded(full1(s), (uint32_t)((it1 / NS1) & 1), ab))) break;
          tc_fence_after();
          const uint32_t st = sR1 + (uint32_t)s * stage1;
          const unsigned long long xd = sw128_desc(st + (uint32_t)MB1 * kBlk);
          const int nk = min(4, (a.n - kt * 64 + 15) >> 4);
          for (int b = 0; b < MB1; ++b) {
            const unsigned long long ad = sw128_desc(st + (uint32_t)b * kBlk);
#pragma unroll
            for (int kk = 0; kk < 4; ++kk)
              if (kk < nk)
                tc_mma(tmem + (uint32_t)(b * a.N1), ad + 2u * kk, xd + 2u * kk, idesc1, (kt > 0 || kk > 0) ? 1u : 0u);
          }
          tc_commit(empty1(s));
        }
        if (!ok) break;
        tc_commit(d1full);
        // step 2: D2[b] = W2 block b . T^T over the K tiles of q, T in shared memory
        if (!(ok = wait_bounded(tready, (uint32_t)(i & 1), ab))) break;
        tc_fence_after();
        for (int b = 0; ok && b < MB2; ++b) {
          for (int kt = 0; ok && kt < a.KT2; ++kt, ++it2) {
            const int s = it2 % NS2;
            if (!(ok = wait_bounded(full2(s), (uint32_t)((it2 / NS2) & 1), ab))) break;
            tc_fence_after();
            const unsigned long long ad = sw128_desc(sR2 + (uint32_t)s * kBlk);
            const unsigned long long td = sw128_desc(sT + (uint32_t)kt * (uint32_t)MB1 * kBlk);
            const int nk = min(4, (a.q - kt * 64 + 15) >> 4);
#pragma unroll
            for (int kk = 0; kk < 4; ++kk)
              if (kk < nk)
                tc_mma(tmem + (uint32_t)(b * a.N2), ad + 2u * kk, td + 2u * kk, idesc2, (kt > 0 || kk > 0) ? 1u : 0u);
            tc_commit(empty2(s));
          }
          if (ok) tc_commit(d2full0 + 8u * (uint32_t)b);
        }
        if (ok) tc_commit(tfree);
      }
      tc_commit(drain);  // every MMA this thread issued is complete once `drain` fires
      const unsigned long long t0 = gtimer();
      while (!mbar_try_wait(drain, 0) && gtimer() - t0 < kWaitLimitNs) {
      }
    }
    __syncwarp();
  } else {
    // ---------------- epilogue: warp (quadrant q4, share h) takes the 16-column chunks h*16 + 64 j
    const int q4 = warp & 3, h = (warp - 2) >> 2;
    BoxEmitter<OutT> em{sO + (uint32_t)(warp - 2) * (uint32_t)a.stg * kOB, a.stg};
    const float zs = (a.last && a.shift_src) ? ldexpf(1.0f, a.sG - *a.shift_src) : 1.0f;
    bool ok = true;
    for (int i = 0; ok && i < nmine; ++i) {
      const int p = (int)blockIdx.x + i * (int)gridDim.x;
      // step-1 drain: T[n'][q] = round(D1[n'][q]), K-major, 128-byte swizzle (piece k of row r at k ^ (r % 8))
      if (!(ok = __all_sync(0xffffffffu, wait_bounded(d1full, (uint32_t)(i & 1), ab)))) break;
      tc_fence_after();
      const int J1 = (a.N1 - h * 16 + 63) / 64;
      for (int b = 0; b < MB1; ++b) {
        const uint32_t tl = tmem + (uint32_t)(b * a.N1) + ((uint32_t)(q4 * 32) << 16);
        const int row = b * 128 + q4 * 32 + lane;
        for (int j = 0; j < J1; j += 2) {
          uint32_t r0[16], r1[16];
          const int c0 = h * 16 + 64 * j, c1 = c0 + 64;
          tc_ld16_issue(tl + (uint32_t)c0, r0);
          if (j + 1 < J1) tc_ld16_issue(tl + (uint32_t)c1, r1);
          tc_ld16_wait(r0);
          if (j + 1 < J1) tc_ld16_wait(r1);
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            if (u == 1 && j + 1 >= J1) break;
            const int c = u ? c1 : c0;
            float v[16];
#pragma unroll
            for (int k = 0; k < 16; ++k) v[k] = __uint_as_float(u ? r1[k] : r0[k]);
            uint32_t pk[8];
            pack16<InT>(v, pk);
            const uint32_t rowa = sT + (uint32_t)(c >> 6) * (uint32_t)MB1 * kBlk + (uint32_t)row * 128u;
            const uint32_t p0 = (uint32_t)((c & 63) >> 3);
#pragma unroll
            for (int k = 0; k < 2; ++k)
              asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(rowa + (((p0 + k) ^ (uint32_t)(row & 7)) << 4)),
                           "r"(pk[4 * k]), "r"(pk[4 * k + 1]), "r"(pk[4 * k + 2]), "r"(pk[4 * k + 3])
                           : "memory");
          }
        }
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // T (generic writes) -> tensor core reads
      tc_fence_before();
      mbar_arrive(tready);
      // step-2 drain: output rows m = q' (or q), 16 consecutive columns per chunk.  The last launch of a
      // solve reads R~ (this thread's row, its chunks of the block) into registers before it waits for
      // the accumulator, so the loads overlap the MMAs.
      const int J2 = (a.N2 - h * 16 + 63) / 64;  // chunks of this warp per block (at most 4)
      uint4 rpre[4][2];
      auto prefetch = [&](int b) {
        if constexpr (FINAL) {
          const int m = b * 128 + q4 * 32 + lane;
#pragma unroll
          for (int j = 0; j < 4; ++j)
            if (j < J2 && m < a.q) {
              const uint4* rp =
                  reinterpret_cast<const uint4*>(a.Rt + ((long long)p * a.q + m) * a.rpitch + h * 16 + 64 * j);
              rpre[j][0] = __ldg(rp);
              rpre[j][1] = __ldg(rp + 1);
            }
        }
      };
      for (int b = 0; ok && b < MB2; ++b) {
        prefetch(b);
        if (!(ok = __all_sync(0xffffffffu, wait_bounded(d2full0 + 8u * (uint32_t)b, (uint32_t)(i & 1), ab)))) break;
        tc_fence_after();
        const uint32_t tl = tmem + (uint32_t)(b * a.N2) + ((uint32_t)(q4 * 32) << 16);
        const int m0 = b * 128 + q4 * 32;
        const int m = m0 + lane;
        auto process = [&](int c, const uint32_t (&r)[16], const uint4 (&rw4)[2]) {
          float v[16];
#pragma unroll
          for (int k = 0; k < 16; ++k) v[k] = __uint_as_float(r[k]);
          if (a.last) {
#pragma unroll
            for (int k = 0; k < 16; ++k) v[k] *= zs;
          }
          if (m0 < a.q) em.put3(&tmO, v, lane, c, m0, p);  // rows past q and columns past n are clipped
          if (FINAL && m < a.q) {
            const uint32_t rw[8] = {rw4[0].x, rw4[0].y, rw4[0].z, rw4[0].w, rw4[1].x, rw4[1].y, rw4[1].z, rw4[1].w};
            float d0 = 0.0f, d1 = 0.0f;
#pragma unroll
            for (int k = 0; k < 8; ++k) {
              const float2 rr = lp2_to_f32<InT>(rw[k]);
              d0 = fmaf(rr.x * rs, v[2 * k], d0);
              d1 = fmaf(rr.y * rs, v[2 * k + 1], d1);
              zmax = fmaxf(zmax, fmaxf(fabsf(v[2 * k]), fabsf(v[2 * k + 1])));
            }
            red0.add(d0 + d1);
            red1.add(((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7])) +
                     (((v[8] + v[9]) + (v[10] + v[11])) + ((v[12] + v[13]) + (v[14] + v[15]))));
          }
        };
#pragma unroll
        for (int jp = 0; jp < 2; ++jp) {  // chunk pairs (2 jp, 2 jp + 1), TMEM loads of a pair issued together
          const int ja = 2 * jp, jb = ja + 1;
          if (ja < J2) {
            uint32_t r0[16], r1[16];
            const int c0 = h * 16 + 64 * ja, c1 = c0 + 64;
            tc_ld16_issue(tl + (uint32_t)c0, r0);
            if (jb < J2) tc_ld16_issue(tl + (uint32_t)c1, r1);
            tc_ld16_wait(r0);
            if (jb < J2) tc_ld16_wait(r1);
            process(c0, r0, rpre[ja]);
            if (jb < J2) process(c1, r1, rpre[jb]);
          }
        }
      }
      if (!ok) break;
      tc_fence_before();
      mbar_arrive(d2empty);
    }
    if (lane == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
  }

  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512u) : "memory");
  }
  if constexpr (FINAL) {
    __shared__ float smax[kFrontalThreads / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) zmax = fmaxf(zmax, __shfl_xor_sync(0xffffffffu, zmax, o));
    if (lane == 0) smax[warp] = zmax;
    __syncthreads();
    if (threadIdx.x == 0) {
      float mx = 0.0f;
      for (int w = 0; w < kFrontalThreads / 32; ++w) mx = fmaxf(mx, smax[w]);
      atomicMax(&a.st->zmax_bits, __float_as_uint(mx));
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

// ------------------------------------------------------------------ tube pair
// The z products of Algorithm 7 on the [t][q'][n'] array viewed as t rows of
// C = q*n columns: each tile is 128 columns of every row.  The data operand is
// MN-major (columns contiguous), loaded as two 64-column TMA boxes per 64-row
// K tile.  PAIR: stage 1 with the forward eigenbasis, the Hadamard step by G
// on the accumulator (null index zeroed, Algorithm 5), rounding into an
// MN-major T in shared memory, stage 2 with the backward eigenbasis (z axis at
// most 128 points: both eigenbases resident).  Otherwise one product (z axis
// up to 256 points), with G applied when apply_g is set.
// TMEM: PAIR D1 at 128*(i&1), D2 at 256 + 128*(i&1); single D at 256*(i&1) + 128*b.
template <class InT, bool PAIR>
__global__ void __launch_bounds__(kSlabThreads, 1)
    k_tube_pair(const __grid_constant__ CUtensorMap tmF, const __grid_constant__ CUtensorMap tmW1,
                const __grid_constant__ CUtensorMap tmW2, const __grid_constant__ CUtensorMap tmO, SlabArgs a) {
  if (a.st && a.st->done) return;
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t* sm = smem_raw + (base - raw);
  const int MBz = a.MBz, KTz = a.KTz, NS = a.NS;
  const uint32_t kStage = (uint32_t)a.KS * 256u;  // KS rows of z x 128 columns (two MN-major atoms)
  constexpr uint32_t kAtomT = 128u * 128u;      // T: one 64-column atom of 128 K rows
  const uint32_t wbytes = (uint32_t)(MBz * KTz) * kBlk;
  const uint32_t sW1 = base;
  const uint32_t sW2 = sW1 + wbytes;
  const uint32_t sT = sW2 + (PAIR ? wbytes : 0u);
  const uint32_t sD = sT + (PAIR ? 2u * 2u * kAtomT : 0u);
  const uint32_t sO = sD + (uint32_t)NS * kStage;
  constexpr uint32_t kOB = 32u * 16u * (uint32_t)sizeof(InT);
  uint8_t* barp = sm + (sO - base) + (size_t)kSlabEpi * 2 * kOB;
  const uint32_t bars = smem_u32(barp);
  auto full = [&](int s) { return bars + 8u * s; };
  auto empty = [&](int s) { return bars + 8u * (NS + s); };
  const uint32_t b0 = bars + 8u * (2 * NS);
  auto d1full = [&](int b) { return b0 + 8u * b; };
  auto d1empty = [&](int b) { return b0 + 16u + 8u * b; };
  auto d2full = [&](int b) { return b0 + 32u + 8u * b; };
  auto d2empty = [&](int b) { return b0 + 48u + 8u * b; };
  auto tready = [&](int b) { return b0 + 64u + 8u * b; };
  const uint32_t vbar = b0 + 80u, drain = b0 + 88u;
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
      mbar_init(d1empty(b), kSlabEpi * 32);
      mbar_init(d2full(b), 1);
      mbar_init(d2empty(b), kSlabEpi * 32);
      mbar_init(tready(b), kSlabEpi * 32);
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
  const int nmine = a.ntiles > (int)blockIdx.x ? (a.ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;

  if (warp == 0) {
    // ---------------- TMA producer: the eigenbases once (they do not depend on the previous launch),
    // then the stages of every column tile (KS rows of z, two 64-column boxes issued together by lanes
    // 0 and 1)
    if (lane == 0) {
      mbar_expect_tx(vbar, (PAIR ? 2u : 1u) * wbytes);
      for (int kt = 0; kt < KTz; ++kt)
        for (int b = 0; b < MBz; ++b) {
          tma_load_2d(sW1 + (uint32_t)(kt * MBz + b) * kBlk, &tmW1, kt * 64, b * 128, vbar);
          if (PAIR) tma_load_2d(sW2 + (uint32_t)(kt * MBz + b) * kBlk, &tmW2, kt * 64, b * 128, vbar);
        }
    }
    asm volatile("griddepcontrol.wait;" ::: "memory");
    int it = 0;
    bool ok = true;
    for (int i = 0; ok && i < nmine; ++i) {
      const int tile = (int)blockIdx.x + i * (int)gridDim.x;
      for (int ks = 0; ks < a.KTs; ++ks, ++it) {
        const int s = it % NS;
        bool w = true;
        if (lane == 0) {
          w = wait_bounded(empty(s), (uint32_t)(((it / NS) & 1) ^ 1), ab);
          if (w) mbar_expect_tx(full(s), kStage);
        }
        if (!(ok = __shfl_sync(0xffffffffu, w, 0))) break;
        if (lane < 2)
          tma_load_2d(sD + (uint32_t)s * kStage + (uint32_t)lane * (kStage / 2), &tmF, tile * kTubeCols + 64 * lane,
                      ks * a.KS, full(s));
      }
    }
    if (!ok && lane == 0) {  // every issued load completes before the CTA may exit
      for (int j = (it > NS ? it - NS : 0); j < it; ++j) {
        const unsigned long long t0 = gtimer();
        while (!mbar_try_wait(full(j % NS), (uint32_t)((j / NS) & 1)) && gtimer() - t0 < kWaitLimitNs) {
        }
      }
      const unsigned long long t0 = gtimer();
      while (!mbar_try_wait(vbar, 0) && gtimer() - t0 < kWaitLimitNs) {
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issuer
      constexpr uint32_t fmt = std::is_same<InT, __half>::value ? 0u : 1u;
      const uint32_t idesc = idesc_f16kind_bmn(128, kTubeCols, fmt);
      bool ok = wait_bounded(vbar, 0, ab);
      int it = 0;
      // stage 1 of tile i: D = W1 . F (data MN-major: K step of 16 rows = +2048 bytes; atoms KS rows apart)
      auto stage1 = [&](int i) {
        const int b = i & 1;
        if (!wait_bounded(d1empty(b), (uint32_t)(((i >> 1) & 1) ^ 1), ab)) return false;
        tc_fence_after();
        const uint32_t dacc = tmem + (PAIR ? (uint32_t)(b * 128) : (uint32_t)(b * 256));
        for (int ks = 0; ks < a.KTs; ++ks, ++it) {
          const int s = it % NS;
          if (!wait_bounded(full(s), (uint32_t)((it / NS) & 1), ab)) return false;
          tc_fence_after();
          const uint32_t sd = sD + (uint32_t)s * kStage;
          const int nk = min(a.KS >> 4, (a.t - ks * a.KS + 15) >> 4);
          for (int mb = 0; mb < MBz; ++mb) {
#pragma unroll
            for (int kk = 0; kk < 8; ++kk)
              if (kk < nk) {
                const int kg = ks * (a.KS >> 4) + kk;  // K step of 16 rows; the eigenbasis K tiles hold 4 of them
                const unsigned long long wd = sw128_desc(sW1 + (uint32_t)((kg >> 2) * MBz + mb) * kBlk) + 2u * (kg & 3);
                tc_mma(dacc + (uint32_t)(mb * 128), wd, mn128_desc(sd + 2048u * kk, kStage / 2, 1024), idesc,
                       (ks > 0 || kk > 0) ? 1u : 0u);
              }
          }
          tc_commit(empty(s));
        }
        tc_commit(d1full(b));
        return true;
      };
      // stage 2 of tile i (PAIR): D2 = W2 . T, T MN-major in shared memory (atoms 16 KB apart)
      auto stage2 = [&](int i) {
        const int b = i & 1;
        if (!wait_bounded(tready(b), (uint32_t)((i >> 1) & 1), ab)) return false;
        if (!wait_bounded(d2empty(b), (uint32_t)(((i >> 1) & 1) ^ 1), ab)) return false;
        tc_fence_after();
        const uint32_t dacc = tmem + 256u + (uint32_t)(b * 128);
        const uint32_t tb = sT + (uint32_t)b * 2u * kAtomT;
        for (int kt = 0; kt < KTz; ++kt) {
          const unsigned long long wd = sw128_desc(sW2 + (uint32_t)kt * kBlk);
          const int nk = min(4, (a.t - kt * 64 + 15) >> 4);
#pragma unroll
          for (int kk = 0; kk < 4; ++kk)
            if (kk < nk)
              tc_mma(dacc, wd + 2u * kk, mn128_desc(tb + (uint32_t)kt * 8192u + 2048u * kk, kAtomT, 1024), idesc,
                     (kt > 0 || kk > 0) ? 1u : 0u);
        }
        tc_commit(d2full(b));
        return true;
      };
      if (PAIR) {
        if (ok && nmine > 0) ok = stage1(0);
        for (int i = 0; ok && i < nmine; ++i) {
          if (i + 1 < nmine && !(ok = stage1(i + 1))) break;
          ok = stage2(i);
        }
      } else {
        for (int i = 0; ok && i < nmine; ++i) ok = stage1(i);
      }
      tc_commit(drain);
      const unsigned long long t0 = gtimer();
      while (!mbar_try_wait(drain, 0) && gtimer() - t0 < kWaitLimitNs) {
      }
    }
    __syncwarp();
  } else {
    // ---------------- epilogue: lanes are z indices, 16 consecutive columns per chunk (one n'-run of one q')
    const int q4 = warp & 3, h = (warp - 2) >> 2;
    BoxEmitter<InT> em{sO + (uint32_t)(warp - 2) * 2u * kOB, 2};
    // G o D for 16 columns c0.. of tile `tile` at row tr (z eigen index): G = 1 / ((lam_x + lam_y) + lam_z)
    // times 2^-sG; zero for the null index and for rows past the z axis
    auto scale_g = [&](float (&v)[16], int tile, int c0, int tr) {
      const int gc = tile * kTubeCols + c0;
      const int jy = gc / a.n, ix = gc - jy * a.n;
      if (tr >= a.t) {
#pragma unroll
        for (int k = 0; k < 16; ++k) v[k] = 0.0f;
        return;
      }
      const float lz = __ldg(a.lamz + tr), ly = __ldg(a.lamy + jy);
      const float4* lx4 = reinterpret_cast<const float4*>(a.lamx + ix);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const float4 l = __ldg(lx4 + k);
        v[4 * k + 0] *= rcp_approx((l.x + ly) + lz) * a.gscale;
        v[4 * k + 1] *= rcp_approx((l.y + ly) + lz) * a.gscale;
        v[4 * k + 2] *= rcp_approx((l.z + ly) + lz) * a.gscale;
        v[4 * k + 3] *= rcp_approx((l.w + ly) + lz) * a.gscale;
      }
      if (a.singular && tr == 0 && gc == 0) v[0] = 0.0f;
    };
    auto ld2 = [&](uint32_t tl, int c0, int c1, uint32_t (&r0)[16], uint32_t (&r1)[16]) {
      tc_ld16_issue(tl + (uint32_t)c0, r0);
      tc_ld16_issue(tl + (uint32_t)c1, r1);
      tc_ld16_wait(r0);
      tc_ld16_wait(r1);
    };
    // PAIR stage 1 of tile i -> T[i & 1] (MN-major: row t' of atom c0/64, piece k at k ^ (t' % 8))
    auto epi1 = [&](int i) {
      const int tile = (int)blockIdx.x + i * (int)gridDim.x;
      const int b = i & 1;
      if (!__all_sync(0xffffffffu, wait_bounded(d1full(b), (uint32_t)((i >> 1) & 1), ab))) return false;
      tc_fence_after();
      const uint32_t tl = tmem + (uint32_t)(b * 128) + ((uint32_t)(q4 * 32) << 16);
      uint32_t r0[16], r1[16];
      const int c0 = h * 16, c1 = c0 + 64;
      ld2(tl, c0, c1, r0, r1);
      tc_fence_before();
      mbar_arrive(d1empty(b));
      const int tr = q4 * 32 + lane;
      const uint32_t tb = sT + (uint32_t)b * 2u * kAtomT + (uint32_t)tr * 128u;
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int c = u ? c1 : c0;
        float v[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) v[k] = __uint_as_float(u ? r1[k] : r0[k]);
        scale_g(v, tile, c, tr);
        uint32_t pk[8];
        pack16<InT>(v, pk);
        const uint32_t rowa = tb + (uint32_t)(c >> 6) * kAtomT;
        const uint32_t p0 = (uint32_t)((c & 63) >> 3);
#pragma unroll
        for (int k = 0; k < 2; ++k)
          asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(rowa + (((p0 + k) ^ (uint32_t)(tr & 7)) << 4)),
                       "r"(pk[4 * k]), "r"(pk[4 * k + 1]), "r"(pk[4 * k + 2]), "r"(pk[4 * k + 3])
                       : "memory");
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_arrive(tready(b));
      return true;
    };
    // output of tile i: the accumulator at TMEM column `col0` + 128 mb, rows t = mb*128 + q4*32 + lane
    auto epi_out = [&](int i, uint32_t full_bar, uint32_t empty_bar, uint32_t col0, int nmb, bool g) {
      const int tile = (int)blockIdx.x + i * (int)gridDim.x;
      if (!__all_sync(0xffffffffu, wait_bounded(full_bar, (uint32_t)((i >> 1) & 1), ab))) return false;
      tc_fence_after();
      for (int mb = 0; mb < nmb; ++mb) {
        const uint32_t tl = tmem + col0 + (uint32_t)(mb * 128) + ((uint32_t)(q4 * 32) << 16);
        uint32_t r0[16], r1[16];
        const int c0 = h * 16, c1 = c0 + 64;
        ld2(tl, c0, c1, r0, r1);
        const int row0 = mb * 128 + q4 * 32;
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const int c = u ? c1 : c0;
          float v[16];
#pragma unroll
          for (int k = 0; k < 16; ++k) v[k] = __uint_as_float(u ? r1[k] : r0[k]);
          if (g) scale_g(v, tile, c, row0 + lane);
          if (row0 < a.t) em.put2(&tmO, v, lane, tile * kTubeCols + c, row0);  // rows past t clipped
        }
      }
      tc_fence_before();
      mbar_arrive(empty_bar);
      return true;
    };
    bool ok = true;
    if (PAIR) {
      for (int i = 0; ok && i < nmine; ++i) {
        ok = epi1(i);
        if (ok && i > 0) ok = epi_out(i - 1, d2full((i - 1) & 1), d2empty((i - 1) & 1), 256u + 128u * ((i - 1) & 1), 1, false);
      }
      if (ok && nmine > 0)
        epi_out(nmine - 1, d2full((nmine - 1) & 1), d2empty((nmine - 1) & 1), 256u + 128u * ((nmine - 1) & 1), 1,
                false);
    } else {
      for (int i = 0; ok && i < nmine; ++i)
        ok = epi_out(i, d1full(i & 1), d1empty(i & 1), 256u * (uint32_t)(i & 1), MBz, a.apply_g != 0);
    }
    if (lane == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
  }

  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512u) : "memory");
  }
}

// ------------------------------------------------------------------ host side
struct SlabLaunch {
  int kind;   // 0 frontal forward, 1 frontal backward (FP32 out), 2 tube pair, 3 single tube pass
  CUtensorMap m0, m1, m2, m3;
  SlabArgs args;
  int grid;
  size_t smem;
};

struct SlabPlan {
  std::vector<SlabLaunch> split;  // z products as two launches
  std::vector<SlabLaunch> fused;  // z products and G as one tube pair (empty when the z axis exceeds 128)
  bool fp16 = false;
  const std::vector<SlabLaunch>& seq(const tpcg_plan* p) const {
    return (p->tc_fuse && !fused.empty()) ? fused : split;
  }
};

int enc(CUtensorMap* map, CUtensorMapDataType dt, int rank, const void* g, const cuuint64_t* dims,
        const cuuint64_t* strides_bytes, const cuuint32_t* box, CUtensorMapSwizzle sw) {
  EncodeTiledFn fn = tma_encoder();
  if (!fn) return -1;
  cuuint32_t estr[3] = {1, 1, 1};
  return fn(map, dt, (cuuint32_t)rank, const_cast<void*>(g), dims, strides_bytes, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
                 CUDA_SUCCESS
             ? 0
             : -1;
}

template <class InT>
int slab_smem_attrs() {
  int bad = 0;
  auto set = [&](const void* f) {
    bad |= cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem) == cudaSuccess ? 0 : 1;
  };
  set((const void*)k_frontal_pair<InT, InT, false>);
  set((const void*)k_frontal_pair<InT, float, false>);
  set((const void*)k_frontal_pair<InT, float, true>);
  set((const void*)k_tube_pair<InT, true>);
  set((const void*)k_tube_pair<InT, false>);
  return bad;
}

template <class InT>
void slab_launch(const SlabLaunch& L, const SlabArgs& a, bool final_pcg, cudaStream_t stream) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)L.grid);
  cfg.blockDim = dim3(L.kind <= 1 ? kFrontalThreads : kSlabThreads);
  cfg.dynamicSmemBytes = L.smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  switch (L.kind) {
    case 0: cudaLaunchKernelEx(&cfg, k_frontal_pair<InT, InT, false>, L.m0, L.m1, L.m2, L.m3, a); break;
    case 1:
      if (final_pcg) cudaLaunchKernelEx(&cfg, k_frontal_pair<InT, float, true>, L.m0, L.m1, L.m2, L.m3, a);
      else cudaLaunchKernelEx(&cfg, k_frontal_pair<InT, float, false>, L.m0, L.m1, L.m2, L.m3, a);
      break;
    case 2: cudaLaunchKernelEx(&cfg, k_tube_pair<InT, true>, L.m0, L.m1, L.m2, L.m3, a); break;
    default: cudaLaunchKernelEx(&cfg, k_tube_pair<InT, false>, L.m0, L.m1, L.m2, L.m3, a); break;
  }
}

}  // namespace

// Smallest positive eigenvalue sum (the FP16 range exponent of G uses it); defined with the per-pass kernels.
int tc_fp16_g_exponent(const tpcg_plan* p);

// The frontal-slice sequence applies to the FP16 and BF16 forms on 3D grids with nx a multiple of 16
// (every slice row and every 16-column chunk aligned), nx, ny, nz <= 256.
bool slab_applicable(const tpcg_plan* p) {
  return (p->prec == TPCG_MIXED_FP16 || p->prec == TPCG_MIXED_BF16) && !p->is2d && p->nx % 16 == 0 && p->nx <= 256 &&
         p->ny <= 256 && p->nz <= 256 && p->nx >= 16;
}

int slab_plan_setup(tpcg_plan* p) {
  if (!slab_applicable(p)) return TPCG_ERR_UNSUPPORTED;
  SlabPlan* sp = new SlabPlan();
  sp->fp16 = (p->prec == TPCG_MIXED_FP16);
  const int n = p->nx, q = p->ny, t = p->nz;
  const CUtensorMapDataType dt = sp->fp16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  const int sG = sp->fp16 ? tc_fp16_g_exponent(p) : 0;
  SlabArgs base{};
  base.n = n;
  base.q = q;
  base.t = t;
  base.sG = sG;
  base.gscale = std::ldexp(1.0f, -sG);
  base.shift_src = sp->fp16 ? &p->d_state->lp_shift_applied : nullptr;
  base.lamx = p->d_lam32[0];
  base.lamy = p->d_lam32[1];
  base.lamz = p->d_lam32[2];
  base.singular = p->singular ? 1 : 0;
  base.Rt = reinterpret_cast<const uint16_t*>(p->d_Rlp);
  base.rpitch = p->pitch16[0];
  base.N = p->N;
  base.err = p->d_err;
  const size_t C = (size_t)q * n;  // columns of a z row of the intermediates ([t][q'][n'], no padding)
  if (p->t_elems < C * (size_t)t) {
    delete sp;
    return TPCG_ERR_UNSUPPORTED;
  }
  int rc = TPCG_OK;
  // frontal pair: in -> out, eigenbases of direction dir; FP32 output for the backward launch
  auto frontal = [&](const void* in, int in_pitch, void* out, int dir, SlabLaunch& L) -> int {
    SlabArgs& a = L.args;
    a = base;
    a.MB1 = (n + 127) / 128;
    a.N1 = ((q + 15) / 16) * 16;
    a.KT1 = (n + 63) / 64;
    a.MB2 = (q + 127) / 128;
    a.N2 = n;
    a.KT2 = (q + 63) / 64;
    a.last = dir;
    L.kind = dir ? 1 : 0;
    const size_t esz = dir ? 4 : 2;
    const uint32_t stage1 = (uint32_t)a.MB1 * kBlk + (uint32_t)a.N1 * 128u;
    const uint32_t tbytes = (uint32_t)a.KT2 * (uint32_t)a.MB1 * kBlk;
    // ring depths and staging boxes that fit, best first: two step-1 stages, then up to four step-2
    // stages, then two staging boxes per epilogue warp, then more step-1 stages
    const size_t barb = 8 * (2 * 4 + 2 * 4 + 7) + 16;
    bool found = false;
    long best = -1;
    for (int ns1 = 1; ns1 <= std::min(a.KT1, 4); ++ns1) {
      const uint32_t reg1 = std::max((uint32_t)ns1 * stage1, tbytes);
      for (int ns2 = 1; ns2 <= std::min(a.MB2 * a.KT2, 4); ++ns2)
        for (int stg = 1; stg <= 2; ++stg) {
          const size_t total = 1024 + (size_t)reg1 + (size_t)ns2 * kBlk + (size_t)kSlabEpi * stg * 32 * 16 * esz + barb;
          const long key = std::min(ns1, 2) * 1000 + ns2 * 100 + stg * 10 + ns1;
          if (total <= (size_t)kMaxSmem && key > best) {
            best = key;
            a.NS1 = ns1;
            a.NS2 = ns2;
            a.reg1 = reg1;
            a.stg = stg;
            L.smem = total;
            found = true;
          }
        }
    }
    if (!found) return TPCG_ERR_UNSUPPORTED;
    const cuuint64_t dX[3] = {(cuuint64_t)n, (cuuint64_t)q, (cuuint64_t)t};
    const cuuint64_t sX[2] = {(cuuint64_t)in_pitch * 2, (cuuint64_t)in_pitch * 2 * q};
    const cuuint32_t bX[3] = {64, (cuuint32_t)a.N1, 1};
    const int lp0 = p->pitch16[0], lp1 = p->pitch16[1];
    const cuuint64_t dA1[3] = {(cuuint64_t)n, (cuuint64_t)n, 1};
    const cuuint64_t sA1[2] = {(cuuint64_t)lp0 * 2, (cuuint64_t)lp0 * 2 * n};
    const cuuint32_t bA1[3] = {64, (cuuint32_t)(a.MB1 * 128), 1};
    const cuuint64_t dA2[2] = {(cuuint64_t)q, (cuuint64_t)q}, sA2[1] = {(cuuint64_t)lp1 * 2};
    const cuuint32_t bA[2] = {64, 128};
    const cuuint64_t dO[3] = {(cuuint64_t)n, (cuuint64_t)q, (cuuint64_t)t};
    const cuuint64_t sO[2] = {(cuuint64_t)n * esz, (cuuint64_t)n * esz * q};
    const cuuint32_t bO[3] = {16, 32, 1};
    if (enc(&L.m0, dt, 3, in, dX, sX, bX, CU_TENSOR_MAP_SWIZZLE_128B) ||
        enc(&L.m1, dt, 3, p->d_Wt16[0][dir], dA1, sA1, bA1, CU_TENSOR_MAP_SWIZZLE_128B) ||
        enc(&L.m2, dt, 2, p->d_Wt16[1][dir], dA2, sA2, bA, CU_TENSOR_MAP_SWIZZLE_128B) ||
        enc(&L.m3, dir ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : dt, 3, out, dO, sO, bO,
            dir ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B))
      return TPCG_ERR_CUDA;
    L.grid = std::max(1, std::min(t, p->num_sms));
    return TPCG_OK;
  };
  // tube launch over [t][C]: kind 2 (pair) or 3 (single pass of direction dir, G when dir == 0)
  auto tube = [&](const void* in, void* out, int kind, int dir, SlabLaunch& L) -> int {
    SlabArgs& a = L.args;
    a = base;
    a.MBz = (t + 127) / 128;
    a.KTz = (t + 63) / 64;
    a.KS = (t <= 64 || t > 128) ? 64 : 128;  // one stage per column tile up to 128 points of z
    a.KTs = (t + a.KS - 1) / a.KS;
    a.ntiles = (int)((C + kTubeCols - 1) / kTubeCols);
    a.apply_g = (kind == 3 && dir == 0) ? 1 : 0;
    L.kind = kind;
    const bool pair = (kind == 2);
    if (pair && a.MBz != 1) return TPCG_ERR_UNSUPPORTED;
    const size_t wbytes = (size_t)a.MBz * a.KTz * kBlk;
    const size_t fixed = 1024 + (pair ? 2 : 1) * wbytes + (pair ? 4 * 128 * 128 : 0) +
                         (size_t)kSlabEpi * 2 * 32 * 16 * 2 + 8 * (2 * 8 + 12) + 16;
    const size_t kStage = (size_t)a.KS * 256;
    if (fixed + 2 * kStage > (size_t)kMaxSmem) return TPCG_ERR_UNSUPPORTED;
    a.NS = (int)std::min<size_t>(6, (kMaxSmem - fixed) / kStage);
    L.smem = fixed + (size_t)a.NS * kStage;
    const cuuint64_t dF[2] = {(cuuint64_t)C, (cuuint64_t)t}, sF[1] = {(cuuint64_t)C * 2};
    const cuuint32_t bF[2] = {64, (cuuint32_t)a.KS};
    const int lp2 = p->pitch16[2];
    const cuuint64_t dW[2] = {(cuuint64_t)t, (cuuint64_t)t}, sW[1] = {(cuuint64_t)lp2 * 2};
    const cuuint32_t bW[2] = {64, 128};
    const cuuint32_t bO[2] = {16, 32};
    const int d1 = pair ? 0 : dir;
    if (enc(&L.m0, dt, 2, in, dF, sF, bF, CU_TENSOR_MAP_SWIZZLE_128B) ||
        enc(&L.m1, dt, 2, p->d_Wt16[2][d1], dW, sW, bW, CU_TENSOR_MAP_SWIZZLE_128B) ||
        enc(&L.m2, dt, 2, p->d_Wt16[2][1], dW, sW, bW, CU_TENSOR_MAP_SWIZZLE_128B) ||
        enc(&L.m3, dt, 2, out, dF, sF, bO, CU_TENSOR_MAP_SWIZZLE_32B))
      return TPCG_ERR_CUDA;
    L.grid = std::max(1, std::min(a.ntiles, p->num_sms));
    return TPCG_OK;
  };
  SlabLaunch L{};
  void* T0 = p->d_T[0];
  void* T1 = p->d_T[1];
  // split: z forward (with G) and z backward as two launches; fused: one tube pair (z axis <= 128)
  if ((rc = frontal(p->d_Rlp, p->pitch16[0], T0, 0, L)) == TPCG_OK) sp->split.push_back(L);
  if (rc == TPCG_OK && (rc = tube(T0, T1, 3, 0, L)) == TPCG_OK) sp->split.push_back(L);
  if (rc == TPCG_OK && (rc = tube(T1, T0, 3, 1, L)) == TPCG_OK) sp->split.push_back(L);
  if (rc == TPCG_OK && (rc = frontal(T0, n, p->d_Z, 1, L)) == TPCG_OK) sp->split.push_back(L);
  if (rc == TPCG_OK && t <= 128) {
    sp->fused.push_back(sp->split[0]);
    if ((rc = tube(T0, T1, 2, 0, L)) == TPCG_OK) sp->fused.push_back(L);
    if (rc == TPCG_OK && (rc = frontal(T1, n, p->d_Z, 1, L)) == TPCG_OK) sp->fused.push_back(L);
  }
  if (rc == TPCG_OK && (sp->fp16 ? slab_smem_attrs<__half>() : slab_smem_attrs<__nv_bfloat16>())) rc = TPCG_ERR_CUDA;
  if (rc != TPCG_OK) {
    delete sp;
    return rc;
  }
  p->slab_state = sp;
  return TPCG_OK;
}

void slab_plan_release(tpcg_plan* p) {
  delete reinterpret_cast<SlabPlan*>(p->slab_state);
  p->slab_state = nullptr;
}

int slab_launches_per_apply(const tpcg_plan* p) {
  const SlabPlan* sp = reinterpret_cast<const SlabPlan*>(p->slab_state);
  return sp ? (int)sp->seq(p).size() : 0;
}

// R~ (the FP16/BF16 copy of R in d_Rlp) -> Z (FP32).  With st the last launch performs the PCG finalize.
int run_precond_slab(const tpcg_plan* p, float* Z, SolveState* st) {
  const SlabPlan* sp = reinterpret_cast<const SlabPlan*>(p->slab_state);
  if (!sp) return TPCG_ERR_UNSUPPORTED;
  const std::vector<SlabLaunch>& seq = sp->seq(p);
  const int ns = (int)seq.size();
  for (int i = 0; i < ns; ++i) {
    const SlabLaunch& L = seq[i];
    SlabArgs a = L.args;
    const bool last = (i == ns - 1);
    if (last && (void*)Z != p->d_Z) return TPCG_ERR_INVALID_ARG;  // the output map names the plan's Z
    a.st = st;
    a.partials = p->d_partials;
    LaunchScope ls(p, kKModeTC);
    if (sp->fp16) slab_launch<__half>(L, a, last && st != nullptr, p->stream);
    else slab_launch<__nv_bfloat16>(L, a, last && st != nullptr, p->stream);
  }
  return TPCG_OK;
}

}  // namespace tpcg
