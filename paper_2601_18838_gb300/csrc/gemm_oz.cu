// Error-free split mode products on tcgen05 (the KPME_BF16X10 arithmetic).
//
// Same contraction as gemm_tc.cu,
//     out[j][n][m] (+)= sum_{(a, f) in pairs(j)} sum_k fac[f][n][k] * in[a][m][k],
// but each operand row is cut into four fixed-point bf16 slices relative to a common
// power of two per row (the splitting of Ozaki, Ogita, Oishi and Rump, "Error-free
// transformations of matrix multiplication", Numer. Algorithms 59, 2012):
//     x = 2^(e-7) (d0 + d1 / 2^8 + d2 / 2^16 + d3 / 2^24),  d_s integers in [-128, 128],
// so every product of leading slices is an integer multiple of one quantum per (row, column)
// and at most 2^14 of them; K <= 256 such products sum to < 2^24 quanta and the float32 MMA
// accumulation of them is exact whatever its rounding.  The leading products go to an
// accumulator D0, the nine products with slice sum 1..3 (at most 2^-8 of D0) to D1.
//
// The input rows come from float32 intermediates (or the float32 hi/lo split of the float64
// charge mesh); converter warps slice them on the fly with the per-row maximum that the
// producing stage recorded (atomicMax over the rows of the consuming stage).  Factors are
// sliced once at plan time and streamed by TMA.  TMEM holds two (D0, D1) pairs so that the
// epilogue drains one Kronecker term while the MMAs of the next run.
// All waits are bounded; a wait that runs out raises the device status word.
#include "kpme_internal.cuh"

namespace kpme {
namespace {

constexpr int kThreads = 320;
constexpr int kBM = 128;
constexpr int kSlices = 4;
constexpr int kProducts = 10;
constexpr int kChunk = 64;                 // k values per chunk = one 128-byte bf16 row
constexpr int kASlice = kBM * 128;         // 16 KB

struct OzParams {
  const void* in;
  int64_t in_bs;
  const float* rowmax_in;
  int64_t rm_in_bs;
  int M, N, Kr;
  int stages, stage_bytes, tmem_cols;
  int mode;          // 0: store out[job][n][m] and the next stage's row maxima; 1: atomicAdd
  float* out;
  int64_t out_bs;
  float* rowmax_out;
  int64_t rm_out_bs;
  const int* start;
  const int2* pairs;
  int n_jobs;
  int nbatch_a;      // batches per slice plane of the pre-sliced A (TMA mode)
  int* status;
};

// products ordered (0,0) | (0,1) (1,0) | (0,2) (1,1) (2,0) | (0,3) (1,2) (2,1) (3,0)
__host__ __device__ constexpr int pa(int p) {
  return p == 0 ? 0 : p == 1 ? 0 : p == 2 ? 1 : p == 3 ? 0 : p == 4 ? 1 : p == 5 ? 2 : p == 6 ? 0 : p == 7 ? 1 : p == 8 ? 2 : 3;
}
__host__ __device__ constexpr int pb(int p) {
  return p == 0 ? 0 : p == 1 ? 1 : p == 2 ? 0 : p == 3 ? 2 : p == 4 ? 1 : p == 5 ? 0 : p == 6 ? 3 : p == 7 ? 2 : p == 8 ? 1 : 0;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag, int* status) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (*abort_flag) return false;
    if (clock64() - t0 > kWaitCycles) {
      *abort_flag = 1;
      atomicExch(status, DEV_TIMEOUT);
      return false;
    }
  }
  return true;
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0, int c1, int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], "
      "[%2];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2)
      : "memory");
}
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}
__host__ __device__ constexpr uint32_t idesc_bf16(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}
__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\ttcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(id), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&h);
}

// 2^k as a float32 (exact): a bit pattern for normal exponents, ldexpf outside.
__device__ __forceinline__ float pow2f(int k) {
  return (k >= -126 && k <= 127) ? __int_as_float((127 + k) << 23) : ldexpf(1.0f, k);
}

// Four fixed-point digits of 8 values scaled by 2^(7 - e): writes slices s = 0..3 of one
// 16-byte group (8 consecutive k) as packed bf16, each slice carrying its own power of two.
// Input: one float32 per value, or a float32 hi/lo pair (hi + lo = the float64 value to
// about 2^-48).  Scaling by a power of two, rint and the subtraction of the digit are exact
// in float32; the lo part joins the first remainder (rounded at 2^-25 of the digit scale,
// below the last digit's resolution).
template <typename TIN>
__device__ __forceinline__ void slice8(const TIN* v, int e, uint4 (&o)[kSlices]) {
  const float up = pow2f(7 - e);
  float t[8];
  float d[kSlices][8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    float th, tl = 0.0f;
    if constexpr (sizeof(TIN) == 8) {
      th = v[i].x * up;
      tl = v[i].y * up;
    } else {
      th = v[i] * up;
    }
    const float d0 = rintf(th);
    d[0][i] = d0;
    t[i] = ((th - d0) + tl) * 256.0f;
  }
#pragma unroll
  for (int s = 1; s < kSlices; ++s) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const float di = rintf(t[i]);
      t[i] = (t[i] - di) * 256.0f;
      d[s][i] = di;
    }
  }
#pragma unroll
  for (int s = 0; s < kSlices; ++s) {
    const float dn = pow2f(e - 7 - 8 * s);
    o[s].x = pack_bf16(d[s][0] * dn, d[s][1] * dn);
    o[s].y = pack_bf16(d[s][2] * dn, d[s][3] * dn);
    o[s].z = pack_bf16(d[s][4] * dn, d[s][5] * dn);
    o[s].w = pack_bf16(d[s][6] * dn, d[s][7] * dn);
  }
}

// Persistent CTA: 10 warps, work items (m-tile, n-tile, job) strided by gridDim.x, every role
// walking the same sequence of (item, pair, 64-wide chunk) so the shared ring counters agree.
//   warp 0      : TMA of the four factor slices per chunk
//   warp 1      : TMEM allocation; lane 0 issues 10 products per 16-wide k step
//   warps 2..5  : converters, one operand row per thread
//   warps 6..9  : epilogue, TMEM lanes 32 (warp % 4) .. + 31, one output row per thread
template <int BN, typename TIN, bool A_TMA>
__global__ void __launch_bounds__(kThreads, 1)
    mp_oz_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, OzParams prm) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  constexpr int kBSlice = BN * 128;
  const int S = prm.stages;
  uint64_t* full_a = reinterpret_cast<uint64_t*>(smem + S * prm.stage_bytes);
  uint64_t* full_b = full_a + S;
  uint64_t* empty = full_b + S;
  uint64_t* acc_full = empty + S;
  uint64_t* acc_empty = acc_full + 2;
  uint32_t* taddr_slot = reinterpret_cast<uint32_t*>(acc_empty + 2);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(taddr_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m_tiles = (prm.M + kBM - 1) / kBM;
  const int n_tiles = prm.N / BN;
  const int n_items = m_tiles * n_tiles * prm.n_jobs;
  const int kchunks = (prm.Kr + kChunk - 1) / kChunk;

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full_a[s], A_TMA ? 1 : 128);
      mbar_init(&full_b[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], 128);
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(taddr_slot)),
                 "r"(prm.tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *taddr_slot;

  auto decode = [&](int w, int& m0, int& n0, int& job) {
    const int per_job = m_tiles * n_tiles;
    job = w / per_job;
    const int rem = w - job * per_job;
    n0 = (rem / m_tiles) * BN;
    m0 = (rem % m_tiles) * kBM;
  };

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- factor slices by TMA ----------------
      int it = 0;
      for (int w = blockIdx.x; w < n_items && !*abort_flag; w += gridDim.x) {
        int m0, n0, job;
        decode(w, m0, n0, job);
        const int p0 = prm.start[job], p1 = prm.start[job + 1];
        for (int p = p0; p < p1; ++p) {
          const int2 pr = prm.pairs[p];
          for (int c = 0; c < kchunks; ++c, ++it) {
            const int s = it % S;
            const uint32_t ph = (uint32_t)(it / S) & 1u;
            if (it >= S && !mbar_wait(&empty[s], ph ^ 1u, abort_flag, prm.status)) break;
            uint8_t* sa = smem + s * prm.stage_bytes;
            uint8_t* sb = sa + kSlices * kASlice;
            if constexpr (A_TMA) {
              mbar_expect_tx(&full_a[s], (uint32_t)(kSlices * kASlice));
#pragma unroll
              for (int a = 0; a < kSlices; ++a)
                tma_load_3d(sa + a * kASlice, &tmA, &full_a[s], c * kChunk, m0, a * prm.nbatch_a + pr.x);
            }
            mbar_expect_tx(&full_b[s], (uint32_t)(kSlices * kBSlice));
#pragma unroll
            for (int b = 0; b < kSlices; ++b)
              tma_load_3d(sb + b * kBSlice, &tmB, &full_b[s], c * kChunk, pr.y * prm.N + n0, b);
          }
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issuer ----------------
      const uint32_t id = idesc_bf16(kBM, BN);
      int it = 0, pc = 0;
      for (int w = blockIdx.x; w < n_items && !*abort_flag; w += gridDim.x) {
        int m0, n0, job;
        decode(w, m0, n0, job);
        const int np = prm.start[job + 1] - prm.start[job];
        for (int pl = 0; pl < np && !*abort_flag; ++pl, ++pc) {
          const int buf = pc & 1;
          if (pc >= 2 && !mbar_wait(&acc_empty[buf], (uint32_t)((pc >> 1) - 1) & 1u, abort_flag, prm.status)) break;
          fence_after();
          const uint32_t d0 = tmem + (uint32_t)(buf * 2 * BN), d1 = d0 + BN;
          for (int c = 0; c < kchunks; ++c, ++it) {
            const int s = it % S;
            const uint32_t ph = (uint32_t)(it / S) & 1u;
            if (!mbar_wait(&full_a[s], ph, abort_flag, prm.status) || !mbar_wait(&full_b[s], ph, abort_flag, prm.status))
              break;
            fence_after();
            int ksteps = (prm.Kr - c * kChunk + 15) / 16;
            ksteps = ksteps > 4 ? 4 : ksteps;
            const uint32_t sa = smem_u32(smem + s * prm.stage_bytes);
            const uint32_t sb = sa + kSlices * kASlice;
            for (int kk = 0; kk < ksteps; ++kk) {
              const bool first = (c == 0 && kk == 0);
#pragma unroll
              for (int p = 0; p < kProducts; ++p) {
                const uint64_t da = sdesc(sa + pa(p) * kASlice + kk * 32);
                const uint64_t db = sdesc(sb + pb(p) * kBSlice + kk * 32);
                if (p == 0)
                  mma_bf16(d0, da, db, id, first ? 0u : 1u);
                else
                  mma_bf16(d1, da, db, id, (first && p == 1) ? 0u : 1u);
              }
            }
            mma_commit(&empty[s]);
          }
          mma_commit(&acc_full[buf]);
        }
      }
    }
  } else if (warp < 6) {
    // ---------------- converters (operand rows sliced on the fly) ----------------
    if constexpr (A_TMA) {
      // the A slices come pre-cut by TMA: nothing to convert
    } else {
    const int r = 32 * (warp - 2) + lane;
    int it = 0;
    bool ok = true;
    for (int w = blockIdx.x; w < n_items && ok; w += gridDim.x) {
      int m0, n0, job;
      decode(w, m0, n0, job);
      const int row = m0 + r;
      const bool valid = row < prm.M;
      const int p0 = prm.start[job], p1 = prm.start[job + 1];
      for (int p = p0; p < p1 && ok; ++p) {
        const int2 pr = prm.pairs[p];
        const TIN* rowp = reinterpret_cast<const TIN*>(prm.in) + (int64_t)pr.x * prm.in_bs + (int64_t)row * prm.Kr;
        int e = 0;
        if (valid) frexpf(prm.rowmax_in[(int64_t)pr.x * prm.rm_in_bs + row], &e);
        for (int c = 0; c < kchunks; ++c, ++it) {
          const int s = it % S;
          const uint32_t ph = (uint32_t)(it / S) & 1u;
          if (it >= S && !mbar_wait(&empty[s], ph ^ 1u, abort_flag, prm.status)) {
            ok = false;
            break;
          }
          uint8_t* sa = smem + s * prm.stage_bytes;
          const int kc = c * kChunk;
          // all loads of a pass are issued before any use, so one memory latency per pass
          constexpr int kPasses = sizeof(TIN) == 8 ? 2 : 1;
          constexpr int kGroups = 8 / kPasses;
#pragma unroll
          for (int h = 0; h < kPasses; ++h) {
            TIN v[kGroups * 8];
#pragma unroll
            for (int g = 0; g < kGroups; ++g) {
              const int k = kc + 8 * (h * kGroups + g);
              if (valid && k < prm.Kr) {
#pragma unroll
                for (int i = 0; i < 8; i += 16 / (int)sizeof(TIN)) {
                  const float4 x = *reinterpret_cast<const float4*>(rowp + k + i);
                  if constexpr (sizeof(TIN) == 4) {
                    v[8 * g + i] = x.x; v[8 * g + i + 1] = x.y; v[8 * g + i + 2] = x.z; v[8 * g + i + 3] = x.w;
                  } else {
                    v[8 * g + i] = make_float2(x.x, x.y);
                    v[8 * g + i + 1] = make_float2(x.z, x.w);
                  }
                }
              } else {
#pragma unroll
                for (int i = 0; i < 8; ++i) v[8 * g + i] = TIN{};
              }
            }
#pragma unroll
            for (int g = 0; g < kGroups; ++g) {
              const int j = h * kGroups + g;
              uint4 o[kSlices];
              slice8(v + 8 * g, e, o);
              const int off = r * 128 + ((j ^ (r & 7)) << 4);
#pragma unroll
              for (int sl = 0; sl < kSlices; ++sl) *reinterpret_cast<uint4*>(sa + sl * kASlice + off) = o[sl];
            }
          }
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          mbar_arrive(&full_a[s]);
        }
      }
    }
    }
  } else {
    // ---------------- epilogue ----------------
    const int r = 32 * (warp & 3) + lane;
    const uint32_t lane_base = tmem + ((uint32_t)(32 * (warp & 3)) << 16);
    int pc = 0;
    bool ok = true;
    for (int w = blockIdx.x; w < n_items && ok; w += gridDim.x) {
      int m0, n0, job;
      decode(w, m0, n0, job);
      const int row = m0 + r;
      const int np = prm.start[job + 1] - prm.start[job];
      float acc[BN];
#pragma unroll
      for (int c = 0; c < BN; ++c) acc[c] = 0.0f;
      for (int pl = 0; pl < np; ++pl, ++pc) {
        const int buf = pc & 1;
        if (!mbar_wait(&acc_full[buf], (uint32_t)(pc >> 1) & 1u, abort_flag, prm.status)) {
          ok = false;
          break;
        }
        fence_after();
#pragma unroll
        for (int c0 = 0; c0 < BN; c0 += 16) {
          uint32_t a0[16], a1[16];
          tmem_ld16(lane_base + (uint32_t)(buf * 2 * BN + c0), a0);
          tmem_ld16(lane_base + (uint32_t)(buf * 2 * BN + BN + c0), a1);
          tmem_wait_ld();
#pragma unroll
          for (int i = 0; i < 16; ++i) acc[c0 + i] += __uint_as_float(a0[i]) + __uint_as_float(a1[i]);
        }
        fence_before();
        mbar_arrive(&acc_empty[buf]);
      }
      if (!ok || *abort_flag || row >= prm.M) continue;
      if (prm.mode == 1) {
        float* o = prm.out + (int64_t)n0 * prm.M + row;
#pragma unroll
        for (int c = 0; c < BN; ++c) atomicAdd(o + (int64_t)c * prm.M, acc[c]);
      } else {
        float* o = prm.out + (int64_t)job * prm.out_bs + (int64_t)n0 * prm.M + row;
#pragma unroll
        for (int c = 0; c < BN; ++c) o[(int64_t)c * prm.M] = acc[c];
        if (prm.rowmax_out != nullptr) {
          // row maxima of the consuming stage: its rows are (n, row / K) with n the output column
          const int K = prm.Kr;
          const int64_t rows_next = prm.M / K;
          unsigned int* dst = reinterpret_cast<unsigned int*>(prm.rowmax_out + (int64_t)job * prm.rm_out_bs) +
                              (int64_t)n0 * rows_next + row / K;
          if ((K % 32) == 0) {
#pragma unroll
            for (int c = 0; c < BN; ++c) {
              const unsigned int mx = __reduce_max_sync(0xffffffffu, __float_as_uint(fabsf(acc[c])));
              if (lane == 0) atomicMax(dst + (int64_t)c * rows_next, mx);
            }
          } else {
#pragma unroll
            for (int c = 0; c < BN; ++c) atomicMax(dst + (int64_t)c * rows_next, __float_as_uint(fabsf(acc[c])));
          }
        }
      }
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 1) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(prm.tmem_cols) : "memory");
  }
}

// Row slicer: every row of K contiguous values (float32, or float64 read as a float32 hi/lo
// pair) is cut into four fixed-point bf16 slices relative to the power of two above its own
// maximum; slice s of row r of batch b goes to out[(s * nbatch + b) * rows + r][k].  One warp
// per row.
template <typename TIN>
__global__ void slice_rows_kernel(const TIN* __restrict__ in, int64_t rows_total, int64_t rows_per_batch, int nbatch,
                                  int K, __nv_bfloat16* __restrict__ out) {
  const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= rows_total) return;
  const TIN* row = in + w * K;
  float m = 0.0f;
  for (int k = lane; k < K; k += 32) {
    if constexpr (sizeof(TIN) == 8) {
      m = fmaxf(m, fabsf((float)row[k]));
    } else {
      m = fmaxf(m, fabsf(row[k]));
    }
  }
  // float32 of a float64 value rounds to nearest: the exponent bound still holds
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  int e = 0;
  frexpf(m, &e);
  const float up = pow2f(7 - e);
  const int64_t b = w / rows_per_batch, r = w - b * rows_per_batch;
  const int64_t plane = (int64_t)nbatch * rows_per_batch * K;
  __nv_bfloat16* o = out + (b * rows_per_batch + r) * K;
  for (int k = lane; k < K; k += 32) {
    float th, tl = 0.0f;
    if constexpr (sizeof(TIN) == 8) {
      const double x = row[k];
      const float h = (float)x;
      th = h * up;
      tl = (float)(x - (double)h) * up;
    } else {
      th = row[k] * up;
    }
    float d = rintf(th);
    float t = ((th - d) + tl) * 256.0f;
    o[k] = __float2bfloat16_rn(d * pow2f(e - 7));
#pragma unroll
    for (int s = 1; s < kSlices; ++s) {
      d = rintf(t);
      t = (t - d) * 256.0f;
      o[s * plane + k] = __float2bfloat16_rn(d * pow2f(e - 7 - 8 * s));
    }
  }
}

template <int BN, typename TIN, bool A_TMA>
cudaError_t launch_bn(cudaStream_t st, const CUtensorMap* tmA, const CUtensorMap* tmB, const OzParams& prm, dim3 grid,
                      int smem) {
  auto kern = mp_oz_kernel<BN, TIN, A_TMA>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  kern<<<grid, kThreads, smem, st>>>(*tmA, *tmB, prm);
  return cudaGetLastError();
}

template <int BN>
cudaError_t launch_mode(const OzArgs& a, cudaStream_t st, const OzParams& prm, dim3 grid, int smem) {
  if (a.tmA) return launch_bn<BN, float, true>(st, a.tmA, a.tmB, prm, grid, smem);
  return launch_bn<BN, float, false>(st, a.tmB, a.tmB, prm, grid, smem);
}

}  // namespace

int oz_stage_bytes(int bn) { return kSlices * kASlice + kSlices * bn * 128; }
int oz_smem_bytes(int bn, int stages) { return stages * oz_stage_bytes(bn) + 1024 + 256; }

cudaError_t launch_mp_oz(kpme_plan_t P, const OzArgs& a) {
  OzParams prm{};
  prm.in = a.in;
  prm.in_bs = a.in_bs;
  prm.rowmax_in = a.rowmax_in;
  prm.rm_in_bs = a.rm_in_bs;
  prm.M = a.M;
  prm.N = a.N;
  prm.Kr = a.Kr;
  prm.stages = P->tc_stages;
  prm.stage_bytes = oz_stage_bytes(P->tc_bn);
  int cols = 32;
  while (cols < 4 * P->tc_bn) cols <<= 1;
  prm.tmem_cols = cols;
  prm.mode = a.mode;
  prm.out = a.out;
  prm.out_bs = a.out_bs;
  prm.rowmax_out = a.rowmax_out;
  prm.rm_out_bs = a.rm_out_bs;
  prm.start = a.jobs->d_start;
  prm.pairs = a.jobs->d_pairs;
  prm.n_jobs = a.jobs->n_jobs;
  prm.nbatch_a = a.nbatch_a;
  prm.status = P->d_status;
  const int smem = oz_smem_bytes(P->tc_bn, P->tc_stages);
  const int items = ((a.M + kBM - 1) / kBM) * (a.N / P->tc_bn) * a.jobs->n_jobs;
  dim3 grid(items < P->sm_count ? items : P->sm_count);
  switch (P->tc_bn) {
    case 32: return launch_mode<32>(a, P->stream, prm, grid, smem);
    case 48: return launch_mode<48>(a, P->stream, prm, grid, smem);
    case 64: return launch_mode<64>(a, P->stream, prm, grid, smem);
    case 96: return launch_mode<96>(a, P->stream, prm, grid, smem);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_slice_rows(kpme_plan_t P, const void* in, bool in_double, int64_t rows_per_batch, int nbatch,
                              int K, void* out) {
  const int threads = 256;
  const int64_t rows = rows_per_batch * nbatch;
  const int64_t blocks = (rows * 32 + threads - 1) / threads;
  if (in_double)
    slice_rows_kernel<double><<<(unsigned)blocks, threads, 0, P->stream>>>((const double*)in, rows, rows_per_batch,
                                                                          nbatch, K, (__nv_bfloat16*)out);
  else
    slice_rows_kernel<float><<<(unsigned)blocks, threads, 0, P->stream>>>((const float*)in, rows, rows_per_batch,
                                                                         nbatch, K, (__nv_bfloat16*)out);
  return cudaGetLastError();
}

}  // namespace kpme
