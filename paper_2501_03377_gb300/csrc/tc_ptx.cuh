// Inline-PTX building blocks of the tensor-core kernels (tcgen05 MMA and TMEM,
// TMA bulk tensor copies, mbarriers) shared by the mode-product kernels.
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cstdint>
#include <type_traits>

#include "tpcg_dev.cuh"

namespace tpcg {
namespace tcx {

constexpr unsigned long long kWaitLimitNs = 2000000000ull;  // 2 s
constexpr int kMaxSmem = 232448 - 1024;  // opt-in limit minus room for static shared memory (560 B used)
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

struct Abort {
  volatile int* flag;  // shared
  int* err;            // global error word
  SolveState* st;
};

// Bounded wait for the phase of parity `parity` to complete.
__device__ __forceinline__ bool wait_bounded(uint32_t bar, uint32_t parity, const Abort& ab) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = gtimer();
  for (;;) {
    if (mbar_try_wait(bar, parity)) return true;
    if (*ab.flag) return false;
    if (gtimer() - t0 > kWaitLimitNs) {
      *ab.flag = 1;
      if (ab.err) atomicExch(ab.err, 1);
      if (ab.st) ab.st->timeout = 1;
      return false;
    }
  }
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int c0, int c1, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          dst),
      "l"((unsigned long long)map), "r"(c0), "r"(c1), "r"(bar)
      : "memory");
}

// TMA store of one staged box (bulk async-group of the issuing thread).
__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, uint32_t src, int c0, int c1) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                   (unsigned long long)map),
               "r"(c0), "r"(c1), "r"(src)
               : "memory");
}
__device__ __forceinline__ void tma_store_3d(const CUtensorMap* map, uint32_t src, int c0, int c1, int c2) {
  asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%1, %2, %3}], [%4];" ::"l"(
                   (unsigned long long)map),
               "r"(c0), "r"(c1), "r"(c2), "r"(src)
               : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tc_mma(uint32_t d, unsigned long long a, unsigned long long b, uint32_t idesc,
                                       uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
// The same MMA with TF32 operands (32-bit containers, K = 8 per instruction), FP32 accumulation.
__device__ __forceinline__ void tc_mma_tf32(uint32_t d, unsigned long long a, unsigned long long b, uint32_t idesc,
                                            uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

// FP32 -> TF32 (10-bit mantissa) with round-to-nearest-even on the bit pattern, kept in an FP32
// container (the tensor core reads the top 19 bits); Inf/NaN unchanged, overflow to Inf.
__device__ __forceinline__ float tf32_rn(float x) {
  const uint32_t b = __float_as_uint(x);
  if ((b & 0x7f800000u) == 0x7f800000u) return x;
  const uint32_t r = b + 0xfffu + ((b >> 13) & 1u);
  return __uint_as_float(r & 0xffffe000u);
}

__device__ __forceinline__ void tc_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

// TMEM -> registers, 16 columns of the thread's lane, in split form for
// software pipelining: issue the load, do other work, then wait.  The wait names the destination registers as in/out
// operands, so the compiler cannot read them before the load has landed.
__device__ __forceinline__ void tc_ld16_issue(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, "
      "[%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
__device__ __forceinline__ void tc_ld16_wait(uint32_t (&r)[16]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                 "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15])
               :
               : "memory");
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, rows of
// 128 bytes, 8-row core groups 1024 bytes apart (tile base 1024-aligned).
__device__ __forceinline__ unsigned long long sw128_desc(uint32_t saddr) {
  unsigned long long d = 0;
  d |= (unsigned long long)((saddr >> 4) & 0x3FFFu);
  d |= (unsigned long long)1 << 16;             // leading-dimension byte offset (unused for swizzled K-major)
  d |= (unsigned long long)(1024 >> 4) << 32;   // stride-dimension byte offset
  d |= (unsigned long long)1 << 46;             // descriptor version
  d |= (unsigned long long)2 << 61;             // 128-byte swizzle
  return d;
}

// Instruction descriptor of kind::f16: A and B both BF16 (fmt 1) or both FP16
// (fmt 0), FP32 D, both K-major.
__host__ __device__ constexpr uint32_t idesc_f16kind(int M, int N, uint32_t fmt) {
  return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// FP32 reciprocal, hardware approximation (max error ~1 ulp): far below the
// FP16/BF16 rounding of the value it scales.
__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// Two 16-bit elements packed in one word (low half first) as FP32; BF16 is the top half of an FP32.
template <class InT>
__device__ __forceinline__ float2 lp2_to_f32(uint32_t w) {
  if constexpr (std::is_same<InT, __half>::value) {
    __half2 h2 = *reinterpret_cast<__half2*>(&w);
    return __half22float2(h2);
  } else {
    return make_float2(__uint_as_float(w << 16), __uint_as_float(w & 0xffff0000u));
  }
}

// Row `lane` of a [32][16] output box staged for a TMA store: FP16/BF16 rows of 32 bytes under the
// 32-byte swizzle (16-byte piece i at i ^ ((lane / 4) % 2)), FP32 rows of 64 bytes under the 64-byte
// swizzle (piece i at i ^ ((lane / 2) % 4)); eight consecutive lanes then cover all 32 banks.
template <class OutT>
__device__ __forceinline__ void stage_row(uint32_t buf, int lane, const float (&x)[16]) {
  if constexpr (sizeof(OutT) == 2) {
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
    const uint32_t row = buf + (uint32_t)lane * 32u;
    const uint32_t sw = (uint32_t)((lane >> 2) & 1);
#pragma unroll
    for (int i = 0; i < 2; ++i)
      asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(row + (((uint32_t)i ^ sw) << 4)), "r"(pk[4 * i]),
                   "r"(pk[4 * i + 1]), "r"(pk[4 * i + 2]), "r"(pk[4 * i + 3])
                   : "memory");
  } else {
    const uint32_t row = buf + (uint32_t)lane * 64u;
    const uint32_t sw = (uint32_t)((lane >> 1) & 3);
#pragma unroll
    for (int i = 0; i < 4; ++i)
      asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(row + (((uint32_t)i ^ sw) << 4)), "f"(x[4 * i]),
                   "f"(x[4 * i + 1]), "f"(x[4 * i + 2]), "f"(x[4 * i + 3])
                   : "memory");
  }
}


__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::
          "r"(dst),
      "l"((unsigned long long)map), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
      : "memory");
}

// Shared-memory matrix descriptor of an MN-major operand (the M or N index contiguous), 128-byte
// swizzle: atoms of 8 K-rows x 64 elements (8 rows of 128 bytes, 1024 bytes), the K-row groups of an
// atom column `sbo` bytes apart and the 64-element atom columns `lbo` bytes apart.  A K step of 16
// elements advances the start address by two row groups.
__device__ __forceinline__ unsigned long long mn128_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  unsigned long long d = 0;
  d |= (unsigned long long)((saddr >> 4) & 0x3FFFu);
  d |= (unsigned long long)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (unsigned long long)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (unsigned long long)1 << 46;
  d |= (unsigned long long)2 << 61;
  return d;
}

// Instruction descriptor of kind::f16 with B MN-major (transpose-B bit); A K-major.
__host__ __device__ constexpr uint32_t idesc_f16kind_bmn(int M, int N, uint32_t fmt) {
  return idesc_f16kind(M, N, fmt) | (1u << 16);
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// cuTensorMapEncodeTiled from the driver (looked up once).
inline EncodeTiledFn tma_encoder() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(ptr);
  }
  return fn;
}

}  // namespace tcx
}  // namespace tpcg
