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
#include "tc_common.cuh"

namespace kpme {
namespace {

using namespace tc;

constexpr int kBM = 128;
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
  int n_jobs, n_pairs;
  int nbatch_a;      // batches per slice plane of the pre-sliced A (TMA mode)
  int* status;
  long long wait_cycles;   // budget of one bounded wait (clock cycles)
};

// Persistent CTA, work items (m-tile, n-tile, job) strided by gridDim.x, every role walking
// the same sequence of (item, pair, 64-wide chunk) so the shared ring counters agree.
//   warp 0            : TMA of the four factor slices per chunk (and of the A slices)
//   warp 1            : TMEM allocation; lane 0 issues 10 products per 16-wide k step
//   warps 2..NCONV+1  : converters (none when TMA brings pre-cut A slices): row 32 (c % 4)
//                       + lane, k groups of part c / 4 of the chunk
//   last 4 warps      : epilogue, TMEM lanes 32 (warp % 4) .. + 31, one output row per thread
template <int NCONV>
constexpr int oz_threads() { return 64 + 32 * NCONV + 128; }

template <int BN, int NCONV, bool A_TMA>
__global__ void __launch_bounds__(oz_threads<NCONV>(), 1)
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
  uint64_t* drain_bar = acc_empty + 2;   // the MMA issuer's last commit, on the way out
  uint32_t* taddr_slot = reinterpret_cast<uint32_t*>(drain_bar + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(taddr_slot + 1);
  const WaitCtl wc{abort_flag, prm.status, prm.wait_cycles};
  // per-warp column maxima of the epilogue (4 x BN)
  unsigned int* red = reinterpret_cast<unsigned int*>(smem + S * prm.stage_bytes + 256);
  // the job tables live in shared memory: every role reads them for every item and pair
  int2* s_pairs = reinterpret_cast<int2*>(red + 4 * BN);
  int* s_start = reinterpret_cast<int*>(s_pairs + prm.n_pairs);
  for (int i = threadIdx.x; i < prm.n_pairs; i += blockDim.x) s_pairs[i] = prm.pairs[i];
  for (int i = threadIdx.x; i <= prm.n_jobs; i += blockDim.x) s_start[i] = prm.start[i];

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m_tiles = (prm.M + kBM - 1) / kBM;
  const int n_tiles = prm.N / BN;
  const int n_items = m_tiles * n_tiles * prm.n_jobs;
  const int kchunks = (prm.Kr + kChunk - 1) / kChunk;

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full_a[s], A_TMA ? 1 : 32 * NCONV);
      mbar_init(&full_b[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], 128);
    }
    mbar_init(drain_bar, 1);
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
    // column tiles innermost: the items that read the same A rows run on neighbouring CTAs at
    // the same time, so the rows come from DRAM once and from L2 for the other column tiles
    n0 = (rem % n_tiles) * BN;
    m0 = (rem / n_tiles) * kBM;
  };

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- factor slices by TMA ----------------
      int it = 0;
      for (int w = blockIdx.x; w < n_items && !*abort_flag; w += gridDim.x) {
        int m0, n0, job;
        decode(w, m0, n0, job);
        const int p0 = s_start[job], p1 = s_start[job + 1];
        for (int p = p0; p < p1; ++p) {
          const int2 pr = s_pairs[p];
          for (int c = 0; c < kchunks; ++c, ++it) {
            const int s = it % S;
            const uint32_t ph = (uint32_t)(it / S) & 1u;
            if (it >= S && !mbar_wait(&empty[s], ph ^ 1u, wc)) break;
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
      // loads in flight land before the CTA leaves (at once unless a wait gave up)
      drain_ring(full_b, S, it, prm.status);
      if constexpr (A_TMA) drain_ring(full_a, S, it, prm.status);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issuer ----------------
      const uint32_t id = idesc_bf16(kBM, BN);
      int it = 0, pc = 0;
      for (int w = blockIdx.x; w < n_items && !*abort_flag; w += gridDim.x) {
        int m0, n0, job;
        decode(w, m0, n0, job);
        const int np = s_start[job + 1] - s_start[job];
        for (int pl = 0; pl < np && !*abort_flag; ++pl, ++pc) {
          const int buf = pc & 1;
          if (pc >= 2 && !mbar_wait(&acc_empty[buf], (uint32_t)((pc >> 1) - 1) & 1u, wc)) break;
          fence_after();
          const uint32_t d0 = tmem + (uint32_t)(buf * 2 * BN), d1 = d0 + BN;
          for (int c = 0; c < kchunks; ++c, ++it) {
            const int s = it % S;
            const uint32_t ph = (uint32_t)(it / S) & 1u;
            if (!mbar_wait(&full_a[s], ph, wc) || !mbar_wait(&full_b[s], ph, wc))
              break;
            fence_after();
            int ksteps = (prm.Kr - c * kChunk + 15) / 16;
            ksteps = ksteps > 4 ? 4 : ksteps;
            // one descriptor per operand and stage; digit planes and k steps are compile-time
            // offsets added to the 14-bit address field (addresses stay below 256 KB: no carry)
            const uint32_t sa = smem_u32(smem + s * prm.stage_bytes);
            const uint64_t da0 = sdesc(sa), db0 = sdesc(sa + kSlices * kASlice);
            auto kstep = [&](int kk, bool first) {
#pragma unroll
              for (int p = 0; p < kProducts; ++p) {
                const uint64_t da = da0 + (uint64_t)((pa(p) * kASlice + kk * 32) >> 4);
                const uint64_t db = db0 + (uint64_t)((pb(p) * kBSlice + kk * 32) >> 4);
                if (p == 0)
                  mma_bf16(d0, da, db, id, first ? 0u : 1u);
                else
                  mma_bf16(d1, da, db, id, (first && p == 1) ? 0u : 1u);
              }
            };
            if (ksteps == 4) {
              kstep(0, c == 0);
              kstep(1, false);
              kstep(2, false);
              kstep(3, false);
            } else {
              for (int kk = 0; kk < ksteps; ++kk) kstep(kk, c == 0 && kk == 0);
            }
            mma_commit(&empty[s]);
          }
          mma_commit(&acc_full[buf]);
        }
      }
      // every MMA issued has completed before tensor memory is released
      mma_commit(drain_bar);
      mbar_drain(drain_bar, 0, prm.status);
    }
  } else if (warp < 2 + NCONV) {
    // ---------------- converters (operand rows sliced on the fly) ----------------
    if constexpr (!A_TMA) {
      constexpr int kParts = NCONV / 4;             // threads per row
      constexpr int kG = (kChunk / 8) / kParts;     // 8-value groups per thread and chunk
      constexpr int kV = 8 * kG;
      const int ci = warp - 2;
      const int r = 32 * (ci % 4) + lane;
      const int j0 = (ci / 4) * kG;
      int it = 0;
      bool ok = true;
      // One unit = (item, pair, 64-wide chunk).  The loads of unit u + 1 are issued before
      // unit u is sliced, so their latency overlaps the wait for a free stage and the slicing.
      float vc[kV];
      float rm_c = 0.0f;
      bool pend = false;
      auto process = [&](const float (&v)[kV], float rm) -> bool {
        const int s = it % S;
        const uint32_t ph = (uint32_t)(it / S) & 1u;
        if (it >= S && !mbar_wait(&empty[s], ph ^ 1u, wc)) return false;
        int e = 0;
        frexpf(rm, &e);
        uint8_t* sa = smem + s * prm.stage_bytes;
#pragma unroll
        for (int jj = 0; jj < kG; ++jj) {
          const int j = j0 + jj;
          uint4 o[kSlices];
          slice8(v + 8 * jj, e, o);
          const int off = r * 128 + ((j ^ (r & 7)) << 4);
#pragma unroll
          for (int sl = 0; sl < kSlices; ++sl) *reinterpret_cast<uint4*>(sa + sl * kASlice + off) = o[sl];
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive(&full_a[s]);
        ++it;
        return true;
      };
      for (int w = blockIdx.x; w < n_items && ok; w += gridDim.x) {
        int m0, n0, job;
        decode(w, m0, n0, job);
        const int row = m0 + r;
        const bool valid = row < prm.M;
        const int p0 = s_start[job], p1 = s_start[job + 1];
        for (int p = p0; p < p1 && ok; ++p) {
          const int2 pr = s_pairs[p];
          const float* rowp = reinterpret_cast<const float*>(prm.in) + (int64_t)pr.x * prm.in_bs + (int64_t)row * prm.Kr;
          const float rm = valid ? prm.rowmax_in[(int64_t)pr.x * prm.rm_in_bs + row] : 0.0f;
          for (int c = 0; c < kchunks; ++c) {
            float vn[kV];
            const int kc = c * kChunk + 8 * j0;
#pragma unroll
            for (int g = 0; g < kV / 4; ++g) {
              const int k = kc + 4 * g;
              float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
              if (valid && k < prm.Kr) x = *reinterpret_cast<const float4*>(rowp + k);
              vn[4 * g] = x.x;
              vn[4 * g + 1] = x.y;
              vn[4 * g + 2] = x.z;
              vn[4 * g + 3] = x.w;
            }
            if (pend && !process(vc, rm_c)) {
              ok = false;
              break;
            }
#pragma unroll
            for (int i = 0; i < kV; ++i) vc[i] = vn[i];
            rm_c = rm;
            pend = true;
          }
        }
      }
      if (pend && ok) process(vc, rm_c);
    }
  } else {
    // ---------------- epilogue ----------------
    // Every epilogue thread runs the same number of items and, where the row maxima are
    // combined in shared memory, the same number of named-barrier syncs, whatever happens
    // to its waits (a failed wait only skips work).
    const int wq = warp & 3;
    const int r = 32 * wq + lane;
    const uint32_t lane_base = tmem + ((uint32_t)(32 * wq) << 16);
    const bool combine = prm.mode == 0 && prm.rowmax_out != nullptr && (prm.Kr % 32) == 0;
    int pc = 0;
    bool ok = true;
    for (int w = blockIdx.x; w < n_items; w += gridDim.x) {
      int m0, n0, job;
      decode(w, m0, n0, job);
      const int row = m0 + r;
      const int np = s_start[job + 1] - s_start[job];
      float acc[BN];
#pragma unroll
      for (int c = 0; c < BN; ++c) acc[c] = 0.0f;
      for (int pl = 0; pl < np; ++pl, ++pc) {
        if (!ok) continue;
        const int buf = pc & 1;
        const bool got = __all_sync(0xffffffffu, mbar_wait(&acc_full[buf], (uint32_t)(pc >> 1) & 1u, wc));
        if (!got) {
          ok = false;
          continue;
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
      const bool live = ok && !*abort_flag && row < prm.M;
      if (prm.mode == 1) {
        if (live) {
          float* o = prm.out + (int64_t)n0 * prm.M + row;
#pragma unroll
          for (int c = 0; c < BN; ++c) atomicAdd(o + (int64_t)c * prm.M, acc[c]);
        }
        continue;
      }
      if (live) {
        float* o = prm.out + (int64_t)job * prm.out_bs + (int64_t)n0 * prm.M + row;
#pragma unroll
        for (int c = 0; c < BN; ++c) o[(int64_t)c * prm.M] = acc[c];
      }
      if (prm.rowmax_out == nullptr) continue;
      // Row maxima of the consuming stage: its row (n, row / K) spans K consecutive rows of
      // this output column n, so the maximum combines lanes, warps and (for K > 128) tiles.
      const int K = prm.Kr;
      const int64_t rows_next = prm.M / K;
      unsigned int* dst = reinterpret_cast<unsigned int*>(prm.rowmax_out + (int64_t)job * prm.rm_out_bs) +
                          (int64_t)n0 * rows_next;
      if (combine) {
        // warp maxima per column, column c kept by lane c % 32
        constexpr int kJ = (BN + 31) / 32;
        unsigned int mx[kJ];
#pragma unroll
        for (int j = 0; j < kJ; ++j) mx[j] = 0u;
#pragma unroll
        for (int c = 0; c < BN; ++c) {
          const unsigned int m = __reduce_max_sync(0xffffffffu, live ? __float_as_uint(fabsf(acc[c])) : 0u);
          if ((c & 31) == lane) mx[c >> 5] = m;
        }
#pragma unroll
        for (int j = 0; j < kJ; ++j)
          if (32 * j + lane < BN) red[wq * BN + 32 * j + lane] = mx[j];
        asm volatile("bar.sync 1, 128;" ::: "memory");
        // the first warp of each consuming row in this tile combines and publishes
        const int g = (m0 + 32 * wq) / K;
        const bool leader = wq == 0 || (m0 + 32 * (wq - 1)) / K != g;
        if (leader && m0 + 32 * wq < prm.M) {
#pragma unroll
          for (int j = 0; j < kJ; ++j) {
            const int c = 32 * j + lane;
            if (c >= BN) continue;
            unsigned int v = red[wq * BN + c];
            for (int w2 = wq + 1; w2 < 4 && (m0 + 32 * w2) / K == g; ++w2) v = max(v, red[w2 * BN + c]);
            if (v != 0u) atomicMax(dst + (int64_t)c * rows_next + g, v);
          }
        }
        asm volatile("bar.sync 1, 128;" ::: "memory");
      } else if ((K % 16) == 0 && K >= 32) {
        // K not a multiple of 32: a warp's 32 rows fall into at most two consuming rows
        // glo and glo + 1; one masked warp maximum per part and column, kept by lane c % 32,
        // published 32 columns per instruction
        constexpr int kJ = (BN + 31) / 32;
        const int glo = (m0 + 32 * wq) / K;
        const bool hi = (row / K) != glo;
        const bool two = __any_sync(0xffffffffu, hi);
        unsigned int mlo[kJ], mhi[kJ];
#pragma unroll
        for (int j = 0; j < kJ; ++j) mlo[j] = mhi[j] = 0u;
#pragma unroll
        for (int c = 0; c < BN; ++c) {
          const unsigned int v = live ? __float_as_uint(fabsf(acc[c])) : 0u;
          const unsigned int a = __reduce_max_sync(0xffffffffu, hi ? 0u : v);
          const unsigned int b = two ? __reduce_max_sync(0xffffffffu, hi ? v : 0u) : 0u;
          if ((c & 31) == lane) {
            mlo[c >> 5] = a;
            mhi[c >> 5] = b;
          }
        }
        if (m0 + 32 * wq < prm.M) {
#pragma unroll
          for (int j = 0; j < kJ; ++j) {
            const int c = 32 * j + lane;
            if (c >= BN) continue;
            if (mlo[j] != 0u) atomicMax(dst + (int64_t)c * rows_next + glo, mlo[j]);
            if (mhi[j] != 0u) atomicMax(dst + (int64_t)c * rows_next + glo + 1, mhi[j]);
          }
        }
      } else if (live) {
#pragma unroll
        for (int c = 0; c < BN; ++c) atomicMax(dst + (int64_t)c * rows_next + row / K, __float_as_uint(fabsf(acc[c])));
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

template <int BN, int NCONV, bool A_TMA>
cudaError_t launch_bn(cudaStream_t st, const CUtensorMap* tmA, const CUtensorMap* tmB, const OzParams& prm, dim3 grid,
                      int smem) {
  auto kern = mp_oz_kernel<BN, NCONV, A_TMA>;
  cudaError_t e = raise_smem_cap(reinterpret_cast<const void*>(kern));
  if (e != cudaSuccess) return e;
  kern<<<grid, oz_threads<NCONV>(), smem, st>>>(*tmA, *tmB, prm);
  return cudaGetLastError();
}

// pre-cut A by TMA: no converter warps; float32 A: 8 converter warps (4 for BN = 96, whose
// epilogue needs the registers)
template <int BN>
cudaError_t launch_mode(const OzArgs& a, cudaStream_t st, const OzParams& prm, dim3 grid, int smem) {
  if (a.tmA) return launch_bn<BN, 0, true>(st, a.tmA, a.tmB, prm, grid, smem);
  return launch_bn<BN, (BN <= 64 ? 8 : 4), false>(st, a.tmB, a.tmB, prm, grid, smem);
}

}  // namespace

int oz_stage_bytes(int bn) { return kSlices * kASlice + kSlices * bn * 128; }
int oz_smem_bytes(int bn, int stages) { return stages * oz_stage_bytes(bn) + 1024 + 256 + 4 * bn * 4; }

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
  prm.wait_cycles = P->wait_cycles;
  prm.n_pairs = (int)a.jobs->h_pairs.size();
  const int smem = oz_smem_bytes(P->tc_bn, P->tc_stages) + prm.n_pairs * (int)sizeof(int2) +
                   (prm.n_jobs + 1) * (int)sizeof(int);
  if (smem > 227 * 1024) return cudaErrorInvalidValue;
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
