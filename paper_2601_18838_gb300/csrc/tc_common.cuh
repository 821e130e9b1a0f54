// Device helpers shared by the tcgen05 kernels of the error-free split (gemm_oz.cu,
// gemm_ozt.cu): mbarrier waits with an iteration budget, TMA tile loads, shared-memory
// matrix descriptors (128-byte swizzle, K-major), the bf16 MMA with accumulators in tensor
// memory, tensor-memory loads and stores, and the fixed-point digit cut.
#pragma once
#include "kpme_internal.cuh"

namespace kpme {
namespace tc {

constexpr int kSlices = 4;
constexpr int kProducts = 10;

// products ordered (0,0) | (0,1) (1,0) | (0,2) (1,1) (2,0) | (0,3) (1,2) (2,1) (3,0)
static __host__ __device__ constexpr int pa(int p) {
  return p == 0 ? 0 : p == 1 ? 0 : p == 2 ? 1 : p == 3 ? 0 : p == 4 ? 1 : p == 5 ? 2 : p == 6 ? 0 : p == 7 ? 1 : p == 8 ? 2 : 3;
}
static __host__ __device__ constexpr int pb(int p) {
  return p == 0 ? 0 : p == 1 ? 1 : p == 2 ? 0 : p == 3 ? 2 : p == 4 ? 1 : p == 5 ? 0 : p == 6 ? 3 : p == 7 ? 2 : p == 8 ? 1 : 0;
}

static __device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
static __device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
static __device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
static __device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
// One arrival for a whole warp (the barrier then counts warps, not threads): the lanes' earlier
// shared-memory and tensor-memory work is ordered before lane 0's arrive by __syncwarp.  This
// cuts the serialized updates of a barrier word 32-fold.
static __device__ __forceinline__ void mbar_arrive_warp(uint64_t* bar) {
  __syncwarp();
  if ((threadIdx.x & 31) == 0) mbar_arrive(bar);
}
// A waiting thread is suspended (not polling, so it takes no issue slots from the warps that
// do the work) until the phase completes or this many nanoseconds pass; the caller's cycle
// budget is checked between suspensions.
constexpr uint32_t kSuspendNs = 10000000u;

static __device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity), "r"(kSuspendNs)
      : "memory");
  return ok != 0;
}
// Non-blocking: has the phase with this parity completed?
static __device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// The bounded waits of one CTA share its abort flag (shared memory; set by the first wait that
// gives up, so that every role stops waiting), the device status word and a budget in clock
// cycles per wait (the plan's, kWaitCycles unless fault injection shortens it).
struct WaitCtl {
  volatile int* abort;
  int* status;
  long long budget;
};
// One suspension of mbarrier.try_wait lasts at most kSuspendNs (20 M cycles at 2 GHz); a shorter
// budget is timed with non-blocking polls instead.
constexpr long long kSuspendCycles = 20000000LL;

static __device__ __forceinline__ bool give_up(const WaitCtl& w) {
  *w.abort = 1;
  atomicExch(w.status, DEV_TIMEOUT);
  return false;
}

static __device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, const WaitCtl& w) {
  if (w.budget >= kSuspendCycles) {
    if (mbar_try_wait(bar, parity)) return true;   // already complete: no clock read on this path
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
      if (*w.abort) return false;
      if (clock64() - t0 > w.budget) return give_up(w);
    }
    return true;
  }
  const long long t0 = clock64();
  while (!mbar_test(bar, parity)) {
    if (*w.abort) return false;
    if (clock64() - t0 > w.budget) return give_up(w);
  }
  return true;
}

// A wait on the way out of a CTA that gave up: TMA copies and MMAs already issued complete on
// their own, and they must land before the CTA releases its shared and tensor memory.  The
// abort flag is not consulted; the production budget bounds the wait.
static __device__ __forceinline__ bool mbar_drain(uint64_t* bar, uint32_t parity, int* status) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > kWaitCycles) {
      atomicExch(status, DEV_TIMEOUT);
      return false;
    }
  }
  return true;
}

// The last min(n, stages) loads of a ring of `stages` buffers whose i-th load completes phase
// i / stages of full[i % stages]: each is the latest use of its buffer, so its parity wait is
// unambiguous, and a phase that completed long ago returns at once.
static __device__ __forceinline__ void drain_ring(uint64_t* full, int stages, int n, int* status) {
  for (int i = n > stages ? n - stages : 0; i < n; ++i) mbar_drain(&full[i % stages], (uint32_t)(i / stages) & 1u, status);
}

static __device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0, int c1, int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], "
      "[%2];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2)
      : "memory");
}
static __device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
static __device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
static __device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}
static __host__ __device__ constexpr uint32_t idesc_bf16(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}
static __device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\ttcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(id), "r"(acc)
      : "memory");
}
static __device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}
static __device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
static __device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

static __device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16};" ::"r"(taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]),
      "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
      : "memory");
}
static __device__ __forceinline__ void tmem_st4(uint32_t taddr, uint4 r) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};" ::"r"(taddr), "r"(r.x), "r"(r.y),
               "r"(r.z), "r"(r.w)
               : "memory");
}
static __device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
// D (tensor memory) (+)= A (tensor memory, lanes = rows, two bf16 per column) x B (shared memory)
static __device__ __forceinline__ void mma_bf16_ta(uint32_t d, uint32_t a_tmem, uint64_t b, uint32_t id, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\ttcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}\n" ::"r"(d),
      "r"(a_tmem), "l"(b), "r"(id), "r"(acc)
      : "memory");
}

static __device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&h);
}

// 2^k as a float32 (exact): a bit pattern for normal exponents, ldexpf outside.
static __device__ __forceinline__ float pow2f(int k) {
  return (k >= -126 && k <= 127) ? __int_as_float((127 + k) << 23) : ldexpf(1.0f, k);
}

// Four fixed-point digits of 8 float32 values relative to 2^e (|v| < 2^e): slice s holds
// d_s 2^(e - 7 - 8s) with integers d_s in [-128, 128], written as packed bf16 (exact: at most
// 8 significant bits).  Each digit is taken by rounding the running remainder to a multiple
// of q_s = 2^(e - 7 - 8s) with the add-and-subtract of C_s = 1.5 * 2^(e + 16 - 8s): for
// |r| < 2^(e + 15 - 8s) the float32 sum r + C_s rounds (to nearest, ties to even) onto the
// grid of q_s, so (r + C_s) - C_s is round(r / q_s) q_s exactly and r - that is exact too.
// The digits equal those of rint(r / q_s) at each step.  Exponents whose C_s would leave the
// normal float32 range take the same steps with rintf.
static __device__ __forceinline__ float magic15(int k) { return __int_as_float(((127 + k) << 23) | (1 << 22)); }

// Two float32 lanes per instruction (sm_100 packed add / subtract, round to nearest even in
// each lane): the same operations as two scalar FADDs, at half the instruction count.
static __device__ __forceinline__ uint64_t f2add(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
static __device__ __forceinline__ uint64_t f2sub(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
static __device__ __forceinline__ uint64_t f2pack(float lo, float hi) {
  return (uint64_t)__float_as_uint(lo) | ((uint64_t)__float_as_uint(hi) << 32);
}
static __device__ __forceinline__ uint32_t bf16x2_of(uint64_t h) {
  return pack_bf16(__uint_as_float((uint32_t)h), __uint_as_float((uint32_t)(h >> 32)));
}

static __device__ __forceinline__ void slice8(const float* v, int e, uint4 (&o)[kSlices]) {
  if (e + 16 <= 127 && e - 8 >= -126) {
    uint64_t C[kSlices];
#pragma unroll
    for (int sl = 0; sl < kSlices; ++sl) {
      const float c = magic15(e + 16 - 8 * sl);
      C[sl] = f2pack(c, c);
    }
    uint32_t w[kSlices][4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      uint64_t r = f2pack(v[2 * i], v[2 * i + 1]);
#pragma unroll
      for (int sl = 0; sl < kSlices; ++sl) {
        const uint64_t h = f2sub(f2add(r, C[sl]), C[sl]);
        if (sl + 1 < kSlices) r = f2sub(r, h);
        w[sl][i] = bf16x2_of(h);
      }
    }
#pragma unroll
    for (int sl = 0; sl < kSlices; ++sl) o[sl] = make_uint4(w[sl][0], w[sl][1], w[sl][2], w[sl][3]);
    return;
  }
  float h[kSlices][8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    float r = v[i];
#pragma unroll
    for (int sl = 0; sl < kSlices; ++sl) {
      const float q = ldexpf(1.0f, e - 7 - 8 * sl);
      h[sl][i] = rintf(r / q) * q;
      r = r - h[sl][i];
    }
  }
#pragma unroll
  for (int sl = 0; sl < kSlices; ++sl) {
    o[sl].x = pack_bf16(h[sl][0], h[sl][1]);
    o[sl].y = pack_bf16(h[sl][2], h[sl][3]);
    o[sl].z = pack_bf16(h[sl][4], h[sl][5]);
    o[sl].w = pack_bf16(h[sl][6], h[sl][7]);
  }
}

}  // namespace tc
}  // namespace kpme
