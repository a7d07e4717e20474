// Fifth-generation tensor-core building blocks (sm_103a, inline PTX).
//
// The dense operator contractions of FR on prisms and tetrahedra (Section
// 2, Eqs. disu and FRfinal: D, M0 and the correction lift applied to many
// elements at once) are small-matrix x many-column products.  These helpers
// run them as tcgen05 MMAs: operands in shared memory in the canonical
// K-major layout without swizzle (8-row x 16-byte core matrices), the FP32
// accumulator in tensor memory (TMEM), one thread issuing the MMAs and
// committing them to an mbarrier that the CTA waits on with a bounded spin.
//
// Precision: kind::tf32 MMAs keep 10 explicit mantissa bits.  The "split"
// form writes each FP32 operand as hi + lo with hi = tf32(x), lo =
// tf32(x - hi) and accumulates hi*hi + hi*lo + lo*hi in FP32, which restores
// ~FP32 accuracy (the lo*lo term is below FP32 resolution).
#pragma once
#include <cstdint>

namespace frgb {

// Canonical K-major layout without swizzle: element (r, k) of an R x K
// operand (R a multiple of 8, K a multiple of 4) lives in the core matrix
// (r / 8, k / 4); core matrices are 128 contiguous bytes (8 rows of 16 B),
// ordered with the K-block index fastest.  Byte offsets of neighbouring core
// matrices: along K (leading dimension) 128 B, along R (stride dimension)
// (K / 4) * 128 B.
__host__ __device__ __forceinline__ int tc_offset(int r, int k, int K) {
  return ((r >> 3) * (K >> 2) + (k >> 2)) * 32 + (r & 7) * 4 + (k & 3);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// shared-memory matrix descriptor (no swizzle)
__device__ __forceinline__ uint64_t tc_desc(const void* p, uint32_t lbo,
                                            uint32_t sbo) {
  const uint32_t a = smem_u32(p);
  uint64_t d = uint64_t((a & 0x3FFFFu) >> 4);
  d |= uint64_t((lbo >> 4) & 0x3FFFu) << 16;
  d |= uint64_t((sbo >> 4) & 0x3FFFu) << 32;
  d |= uint64_t(1) << 46;  // descriptor version
  return d;
}

// Offset (in floats) of element (r, k) of an R-row operand stored K-major
// with the 128-byte swizzle: K is cut into atoms of 32 values; atom a holds
// R rows of 128 B (8-row groups 1024 B apart) and the 16-byte chunk index
// inside a row is XORed with r mod 8.  A warp writing 32 consecutive k of one
// row touches 32 distinct banks.  Atom bases must be 1024-byte aligned.
__host__ __device__ __forceinline__ int sw128_offset(int r, int k, int R) {
  const int a = k >> 5, kk = k & 31;
  return a * R * 32 + r * 32 + ((((kk >> 2) ^ (r & 7))) << 2) + (kk & 3);
}

// descriptor of the 8-value K slice `s` of a 128-byte-swizzled operand
__device__ __forceinline__ uint64_t tc_desc_sw128(const float* base, int R,
                                                  int s) {
  const uint32_t a = smem_u32(base + (s >> 2) * R * 32) + uint32_t(s & 3) * 32u;
  uint64_t d = uint64_t((a & 0x3FFFFu) >> 4);
  d |= uint64_t(1) << 16;             // leading offset: unused when swizzled
  d |= uint64_t(1024 >> 4) << 32;     // 8-row groups 1024 B apart
  d |= uint64_t(1) << 46;             // descriptor version
  d |= uint64_t(2) << 61;             // 128-byte swizzle
  return d;
}

// instruction descriptor: kind::tf32, FP32 accumulator, both operands
// K-major, shape M x N
__host__ __device__ constexpr uint32_t tc_idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | (uint32_t(N >> 3) << 17) |
         (uint32_t(M >> 4) << 24);
}

__device__ __forceinline__ float tf32_hi(float x) {
  uint32_t u;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(x));
  return __uint_as_float(u);
}

// TMEM allocation by one full warp; the address lands in *slot (smem).
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile(
      "tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
          smem_u32(slot)),
      "r"(ncols)
      : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::
                   : "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr),
               "r"(ncols)
               : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// make generic-proxy shared-memory writes visible to the tensor core
__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void tc_mma_tf32(uint32_t dtmem, uint64_t adesc,
                                            uint64_t bdesc, uint32_t idesc,
                                            bool accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(uint32_t(accumulate))
      : "memory");
}

__device__ __forceinline__ void tc_commit(uint64_t* mbar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(mbar))
      : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t* mbar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)),
               "r"(count)
               : "memory");
}

__device__ __forceinline__ void mbar_inval(uint64_t* mbar) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(mbar)) : "memory");
}

// make an initialised mbarrier visible to the asynchronous proxy
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Bounded wait for phase `parity` of an mbarrier: gives up (returns false)
// after `timeout_ns` nanoseconds of wall time or 2^24 polls.
__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, uint32_t parity,
                                          unsigned long long timeout_ns) {
  const unsigned long long t0 = global_ns();
  for (int it = 0; it < (1 << 24); ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(mbar)), "r"(parity)
        : "memory");
    if (done) return true;
    if ((it & 63) == 63) {
      if (global_ns() - t0 > timeout_ns) return false;
      __nanosleep(32);
    }
  }
  return false;
}

// Five 4-column chunks of this thread's TMEM lane (addresses a[0..4]) with a
// single wait; the loads and the wait share one asm statement so that no use
// of the results can be scheduled before the wait.
__device__ __forceinline__ void tmem_ld4x5(const uint32_t a[5], float v[5][4]) {
  uint32_t r[20];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%20];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%4, %5, %6, %7}, [%21];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%8, %9, %10, %11}, [%22];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%12, %13, %14, %15}, [%23];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%16, %17, %18, %19}, [%24];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
        "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]),
        "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(a[4])
      : "memory");
#pragma unroll
  for (int i = 0; i < 5; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) v[i][j] = __uint_as_float(r[4 * i + j]);
}

// 16 consecutive FP32 accumulator columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float v[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, "
      "%8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
        "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]),
        "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// 32 consecutive FP32 accumulator columns of this thread's TMEM lane
// (warp w of a warpgroup owns lanes 32w .. 32w+31)
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float v[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, "
      "%8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, "
      "%23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
        "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]),
        "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
        "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]),
        "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Store x as its TF32 pair (hi, lo) at element (r, k) of a 128-byte-swizzled
// operand of R rows.
__device__ __forceinline__ void put_split(float* hi, float* lo, int R, int r,
                                          int k, float x) {
  const int o = sw128_offset(r, k, R);
  const float h = tf32_hi(x);
  hi[o] = h;
  lo[o] = tf32_hi(x - h);
}

// D (+)= A B^T with A = Ah + Al (canonical K-major, no swizzle, K columns)
// and B = Bh + Bl (128-byte swizzle, R rows), over the 8-wide K slice `sa`
// of A and `sb` of B: three kind::tf32 MMAs, the small terms first.
__device__ __forceinline__ void mma3(uint32_t d, const float* ah,
                                     const float* al, int K, int sa,
                                     const float* bh, const float* bl, int R,
                                     int sb, uint32_t idesc, bool acc) {
  const uint32_t sbo = uint32_t(K / 4) * 128u;
  const uint64_t a_h = tc_desc(ah + sa * 64, 128, sbo);
  const uint64_t a_l = tc_desc(al + sa * 64, 128, sbo);
  const uint64_t b_h = tc_desc_sw128(bh, R, sb);
  const uint64_t b_l = tc_desc_sw128(bl, R, sb);
  tc_mma_tf32(d, a_l, b_h, idesc, acc);
  tc_mma_tf32(d, a_h, b_l, idesc, true);
  tc_mma_tf32(d, a_h, b_h, idesc, true);
}

// Shared-memory operands written by all threads -> visible to the MMA issuer.
__device__ __forceinline__ void tc_sync_for_mma() {
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
}

constexpr unsigned long long kTcTimeoutNs = 500000000ull;  // 0.5 s

// Every thread waits for the MMAs committed to `mbar`; the result is made
// uniform over the CTA.
__device__ __forceinline__ bool tc_wait_all(uint64_t* mbar, uint32_t parity) {
  bool ok = mbar_wait(mbar, parity, kTcTimeoutNs);
  ok = __syncthreads_and(ok) != 0;
  tc_fence_after();
  return ok;
}

}  // namespace frgb
