// Tensor-core mode products on sm_103a: tcgen05.mma with TMEM accumulators, operands staged
// in shared memory by TMA.
//
// Same contraction as gemm_simt.cu (one reshaped Kronecker step of Algorithm 2, stored
// transposed so the contracted index becomes the slowest):
//     out[j][n][m] (+)= sum_{(a, f) in pairs(j)} sum_k fac[f][n][k] * in[a][m][k]
// with each value carried as S bf16 slices (or tf32 hi/lo in float32) and the products of
// slices whose indices sum to at most S - 1 accumulated in one float32 TMEM accumulator.
//
// CTA = 128 threads = 4 warps, one 128 x BN output tile:
//   warp 0 lane 0 : TMA producer (A slices [128 rows x 128 B], B slices [BN rows x 128 B])
//   warp 1        : TMEM allocation; lane 0 issues the MMAs and tcgen05.commit
//   warps 0..3    : epilogue, warp w reads TMEM lanes 32w..32w+31 (rows) with tcgen05.ld
// Shared-memory operands use the canonical K-major 128-byte-swizzle layout written by TMA
// (8-row x 128-byte atoms, stride 1024 B between atoms); the K sub-steps of one 128-byte row
// are addressed by advancing the descriptor start address by 32 bytes.
// Every wait is bounded; a wait that runs out raises the plan's device status word and the
// CTA leaves after releasing its TMEM.
#include "kpme_internal.cuh"

namespace kpme {
namespace {

constexpr int kThreads = 128;
constexpr int kBM = 128;
constexpr int kRowBytes = 128;                      // one swizzle atom row of K
constexpr int kASliceBytes = kBM * kRowBytes;       // 16 KB

struct TcParams {
  int M, N, Kr;
  int nbatchA;
  int bn;             // output columns per CTA (multiple of 16, <= 256)
  int stages;
  int stage_bytes;
  int tmem_cols;
  int elem_bytes;     // 2 (bf16) or 4 (float/tf32)
  int kstep_elems;    // 16 (bf16) or 8 (tf32)
  int mode;           // 0: store slices of out; 1: atomicAdd float
  int64_t out_plane;
  void* out;
  const int* start;
  const int2* pairs;
  int* status;
  long long wait_cycles;   // budget of one bounded wait (clock cycles)
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait: false if the budget runs out or another thread already gave up.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag, int* status,
                                          long long budget) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (*abort_flag) return false;
    if (clock64() - t0 > budget) {
      *abort_flag = 1;
      atomicExch(status, DEV_TIMEOUT);
      return false;
    }
  }
  return true;
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0, int c1,
                                            int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], "
      "[%2];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2)
      : "memory");
}

__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }

// K-major, 128-byte swizzle shared-memory matrix descriptor (sm_100 format).
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);        // start address
  d |= (uint64_t)1 << 16;                          // leading byte offset (unused for SW128 K-major)
  d |= (uint64_t)(1024 >> 4) << 32;                // stride byte offset: 8 rows x 128 B
  d |= (uint64_t)1 << 46;                          // descriptor version
  d |= (uint64_t)2 << 61;                          // SWIZZLE_128B
  return d;
}

// Instruction descriptor: D = F32, A/B = BF16 (kind::f16) or TF32 (kind::tf32), both K-major.
__host__ __device__ constexpr uint32_t idesc(bool tf32, int m, int n) {
  return (1u << 4) | ((tf32 ? 2u : 1u) << 7) | ((tf32 ? 2u : 1u) << 10) | ((uint32_t)(n >> 3) << 17) |
         ((uint32_t)(m >> 4) << 24);
}

template <bool TF32>
__device__ __forceinline__ void mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
  if constexpr (TF32) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(id), "r"(acc)
        : "memory");
  } else {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(id), "r"(acc)
        : "memory");
  }
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ float tf32_rn(float x) {
  uint32_t u = __float_as_uint(x);
  if ((u & 0x7f800000u) == 0x7f800000u) return x;
  u += 0xfffu + ((u >> 13) & 1u);
  u &= 0xffffe000u;
  return __uint_as_float(u);
}

// Slice pairs (a, b) with a + b <= S - 1, listed so that the first 1 / 3 / 6 entries are
// the products of S = 1 / 2 / 3: (0,0) (0,1) (1,0) (0,2) (1,1) (2,0).
__host__ __device__ constexpr int n_prods(int S) { return S == 1 ? 1 : (S == 2 ? 3 : 6); }
__host__ __device__ constexpr int prod_a(int p) { return p == 2 ? 1 : (p == 4 ? 1 : (p == 5 ? 2 : 0)); }
__host__ __device__ constexpr int prod_b(int p) { return p == 1 ? 1 : (p == 3 ? 2 : (p == 4 ? 1 : 0)); }

template <bool TF32, int S>
__global__ void __launch_bounds__(kThreads, 1)
    mp_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, TcParams prm) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + prm.stages * prm.stage_bytes);
  uint64_t* empty = full + prm.stages;
  uint64_t* done = empty + prm.stages;
  uint32_t* taddr_slot = reinterpret_cast<uint32_t*>(done + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(taddr_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * kBM;
  const int n0 = blockIdx.y * prm.bn;
  const int job = blockIdx.z;
  const int bslice_bytes = prm.bn * kRowBytes;

  if (threadIdx.x == 0) {
    for (int s = 0; s < prm.stages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(done, 1);
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

  const int p0 = prm.start[job], p1 = prm.start[job + 1];
  const int chunk_elems = kRowBytes / prm.elem_bytes;
  const int kchunks = (prm.Kr + chunk_elems - 1) / chunk_elems;
  const int total = (p1 - p0) * kchunks;

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer ----------------
    int issued = 0;
    for (int it = 0; it < total; ++it) {
      const int s = it % prm.stages;
      const uint32_t ph = (uint32_t)(it / prm.stages) & 1u;
      if (it >= prm.stages && !mbar_wait(&empty[s], ph ^ 1u, abort_flag, prm.status, prm.wait_cycles)) break;
      if (*abort_flag) break;
      const int2 pr = prm.pairs[p0 + it / kchunks];
      const int kc = (it % kchunks) * chunk_elems;
      uint8_t* st = smem + s * prm.stage_bytes;
      mbar_expect_tx(&full[s], (uint32_t)(S * (kASliceBytes + bslice_bytes)));
#pragma unroll
      for (int a = 0; a < S; ++a) tma_load_3d(st + a * kASliceBytes, &tmA, &full[s], kc, m0, a * prm.nbatchA + pr.x);
#pragma unroll
      for (int b = 0; b < S; ++b)
        tma_load_3d(st + S * kASliceBytes + b * bslice_bytes, &tmB, &full[s], kc, pr.y * prm.N + n0, b);
      ++issued;
    }
    if (*abort_flag) {
      // let copies already in flight land before the CTA releases its shared memory
      for (int it = (issued > prm.stages ? issued - prm.stages : 0); it < issued; ++it) {
        const long long t0 = clock64();
        while (!mbar_try_wait(&full[it % prm.stages], (uint32_t)(it / prm.stages) & 1u) &&
               clock64() - t0 < kWaitCycles) {
        }
      }
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer ----------------
    const uint32_t id = idesc(TF32, kBM, prm.bn);
    bool ok = true;
    for (int it = 0; it < total; ++it) {
      const int s = it % prm.stages;
      const uint32_t ph = (uint32_t)(it / prm.stages) & 1u;
      if (!mbar_wait(&full[s], ph, abort_flag, prm.status, prm.wait_cycles)) {
        ok = false;
        break;
      }
      fence_after();
      const int kc = (it % kchunks) * chunk_elems;
      int ksteps = (prm.Kr - kc + prm.kstep_elems - 1) / prm.kstep_elems;
      ksteps = ksteps > 4 ? 4 : ksteps;
      const uint32_t sa = smem_u32(smem + s * prm.stage_bytes);
      const uint32_t sb = sa + S * kASliceBytes;
      for (int kk = 0; kk < ksteps; ++kk) {
#pragma unroll
        for (int p = 0; p < n_prods(S); ++p) {
          const uint64_t da = sdesc(sa + prod_a(p) * kASliceBytes + kk * 32);
          const uint64_t db = sdesc(sb + prod_b(p) * bslice_bytes + kk * 32);
          mma<TF32>(tmem, da, db, id, (it > 0 || kk > 0 || p > 0) ? 1u : 0u);
        }
      }
      mma_commit(&empty[s]);
    }
    (void)ok;
    mma_commit(done);
    // every MMA issued has completed before tensor memory is released, also when a wait gave
    // up (the abort flag is not consulted here; the production budget bounds the wait)
    {
      const long long t0 = clock64();
      while (!mbar_try_wait(done, 0u) && clock64() - t0 < kWaitCycles) {
      }
    }
  }
  __syncwarp();

  // ---------------- epilogue ----------------
  if (total > 0) mbar_wait(done, 0, abort_flag, prm.status, prm.wait_cycles);
  __syncthreads();   // makes the abort decision uniform before the .sync.aligned TMEM loads
  const bool ok = (total > 0) && !*abort_flag;
  fence_after();
  if (ok) {
    const int row = m0 + warp * 32 + lane;
    const int64_t MN = (int64_t)prm.N * prm.M;
    for (int c0 = 0; c0 < prm.bn; c0 += 16) {
      uint32_t r[16];
      tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, r);
      if (row >= prm.M) continue;
#pragma unroll
      for (int c = 0; c < 16; ++c) {
        const int n = n0 + c0 + c;
        const float v = __uint_as_float(r[c]);
        const int64_t off = (int64_t)n * prm.M + row;
        if (prm.mode == 1) {
          atomicAdd(reinterpret_cast<float*>(prm.out) + off, v);
        } else if constexpr (TF32) {
          float* o = reinterpret_cast<float*>(prm.out) + (int64_t)job * MN + off;
          const float hi = tf32_rn(v);
          o[0] = hi;
          if (S > 1) o[prm.out_plane] = tf32_rn(v - hi);   // the tensor core would truncate it
        } else {
          __nv_bfloat16* o = reinterpret_cast<__nv_bfloat16*>(prm.out) + (int64_t)job * MN + off;
          float rem = v;
#pragma unroll
          for (int s = 0; s < S; ++s) {
            const __nv_bfloat16 h = __float2bfloat16_rn(rem);
            o[s * prm.out_plane] = h;
            rem -= __bfloat162float(h);
          }
        }
      }
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 1) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(prm.tmem_cols)
                 : "memory");
  }
}

// fp32 -> S slices (bf16 round-to-nearest cascade, or tf32 hi / lo in float32)
template <bool TF32, int S, typename TS>
__global__ void split_kernel(const TS* __restrict__ src, void* __restrict__ dst, int64_t count) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
    const double v = (double)src[i];
    if constexpr (TF32) {
      const float hi = tf32_rn((float)v);
      reinterpret_cast<float*>(dst)[i] = hi;
      if (S > 1) reinterpret_cast<float*>(dst)[count + i] = tf32_rn((float)(v - (double)hi));
    } else {
      double rem = v;
#pragma unroll
      for (int s = 0; s < S; ++s) {
        const __nv_bfloat16 h = __double2bfloat16(rem);
        reinterpret_cast<__nv_bfloat16*>(dst)[s * count + i] = h;
        rem -= (double)__bfloat162float(h);
      }
    }
  }
}

template <bool TF32, int S>
cudaError_t launch_t(kpme_plan_t P, const TcArgs& a, TcParams prm, dim3 grid, int smem) {
  auto kern = mp_tc_kernel<TF32, S>;
  cudaError_t e = raise_smem_cap(reinterpret_cast<const void*>(kern));
  if (e != cudaSuccess) return e;
  kern<<<grid, kThreads, smem, P->stream>>>(*a.tmA, *a.tmB, prm);
  return cudaGetLastError();
}

PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &p, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

}  // namespace

int tc_smem_bytes(const PrecInfo& pi, int bn, int stages) {
  const int stage = pi.slices * (kASliceBytes + bn * kRowBytes);
  return stages * stage + 1024 /*alignment*/ + 256 /*barriers*/;
}

bool encode_tmap(kpme_plan_t P, CUtensorMap* map, const void* base, int elem_bytes, bool is_f32, uint64_t dim0,
                 uint64_t dim1, uint64_t dim2, uint32_t box0, uint32_t box1) {
  auto enc = get_encode();
  if (!enc) {
    P->last_error = "cuTensorMapEncodeTiled is not available";
    return false;
  }
  cuuint64_t dims[3] = {dim0, dim1, dim2};
  cuuint64_t strides[2] = {dim0 * elem_bytes, dim0 * dim1 * elem_bytes};
  cuuint32_t box[3] = {box0, box1, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = enc(map, is_f32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3,
                   const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    char buf[128];
    snprintf(buf, sizeof(buf), "cuTensorMapEncodeTiled failed (%d)", (int)r);
    P->last_error = buf;
    return false;
  }
  return true;
}

cudaError_t launch_mp_tc(kpme_plan_t P, const TcArgs& a) {
  const PrecInfo& pi = P->prec;
  TcParams prm{};
  prm.M = a.M;
  prm.N = a.N;
  prm.Kr = a.Kr;
  prm.nbatchA = a.nbatchA;
  prm.bn = P->tc_bn;
  prm.stages = P->tc_stages;
  prm.stage_bytes = pi.slices * (kASliceBytes + prm.bn * kRowBytes);
  int cols = 32;
  while (cols < prm.bn) cols <<= 1;
  prm.tmem_cols = cols;
  prm.elem_bytes = pi.elem_bytes;
  prm.kstep_elems = pi.tf32 ? 8 : 16;
  prm.mode = a.mode;
  prm.out_plane = a.out_plane;
  prm.out = a.out;
  prm.start = a.jobs->d_start;
  prm.pairs = a.jobs->d_pairs;
  prm.status = P->d_status;
  prm.wait_cycles = P->wait_cycles;
  // keep (CTAs per SM) x (TMEM columns) <= 512 by asking for enough shared memory
  int smem = tc_smem_bytes(pi, prm.bn, prm.stages);
  const int max_ctas = 512 / cols;
  const int min_smem = (227 * 1024) / (max_ctas + 1) + 1;
  if (max_ctas < 16 && smem < min_smem) smem = min_smem;
  dim3 grid((a.M + kBM - 1) / kBM, a.N / prm.bn, a.jobs->n_jobs);
  if (pi.tf32) {
    if (pi.slices == 1) return launch_t<true, 1>(P, a, prm, grid, smem);
    return launch_t<true, 2>(P, a, prm, grid, smem);
  }
  if (pi.slices == 1) return launch_t<false, 1>(P, a, prm, grid, smem);
  if (pi.slices == 2) return launch_t<false, 2>(P, a, prm, grid, smem);
  return launch_t<false, 3>(P, a, prm, grid, smem);
}

template <typename TS>
cudaError_t split_t(kpme_plan_t P, const TS* src, void* dst, int64_t count) {
  const PrecInfo& pi = P->prec;
  int grid = (int)((count + 255) / 256);
  if (grid > P->sm_count * 8) grid = P->sm_count * 8;
  if (pi.tf32) {
    if (pi.slices == 1) split_kernel<true, 1, TS><<<grid, 256, 0, P->stream>>>(src, dst, count);
    else split_kernel<true, 2, TS><<<grid, 256, 0, P->stream>>>(src, dst, count);
  } else if (pi.slices == 1) {
    split_kernel<false, 1, TS><<<grid, 256, 0, P->stream>>>(src, dst, count);
  } else if (pi.slices == 2) {
    split_kernel<false, 2, TS><<<grid, 256, 0, P->stream>>>(src, dst, count);
  } else {
    split_kernel<false, 3, TS><<<grid, 256, 0, P->stream>>>(src, dst, count);
  }
  return cudaGetLastError();
}

cudaError_t launch_split(kpme_plan_t P, const void* src, bool src_double, void* dst, int64_t count) {
  if (src_double) return split_t<double>(P, (const double*)src, dst, count);
  return split_t<float>(P, (const float*)src, dst, count);
}

}  // namespace kpme
