// Fused second and third mode products of the SKP for K = 32 and K = 64 (KPME_BF16X10).
//
// For one 128-row tile of Y_i (rows (k3', k1) with k1 fastest, K/... of them per k3') and
// a range of terms t, every term runs both remaining steps of Algorithm 2 on the SM:
//     Z_t = Y_i x_2 B_t      (tile rows (k3', k1), columns k2')
//     Phi += Z_t x_1 A_t     (rows (k2', k3'), contraction over k1, columns k1')
// Z_t never leaves the SM: the epilogue warps drain the first product's accumulators and
// write Z_t transposed (rows (k3', k2'), k1 fastest) into a shared-memory tile; converter
// warps cut each row into four fixed-point bf16 digits with the power of two above the row's
// own maximum (a full row is one thread's 64 values) as the A operand of the second
// product.  Both products use the error-free split of
// gemm_oz.cu / gemm_ozt.cu (ten digit products, exact leading accumulator D0, cross terms
// D1; Ozaki, Ogita, Oishi and Rump, Numer. Algorithms 59, 2012), drained per term.  The
// Phi tile is summed over the item's terms in registers and added to the mesh atomically.
//
// Operands: the Y_i digits (A of step 2) are cut by the converter warps from rows read in
// one go from global memory into a 64 KB shared-memory tile in the MMA's swizzled K-major
// layout; the Z_t digits (A of step 3) go to tensor memory, whose 512 columns hold two
// accumulators (2 BN each, taken by the ops in turn, so the epilogue drains one while the
// tensor pipe fills the other) and two Z_t digit slots (128 each).  The factor digits come
// by TMA.  The tensor pipe alternates step 2 of term j + 1 and step 3 of term j; two MMA
// threads issue the ops of one accumulator each, so one thread's waits overlap the other's
// MMAs; the transposed Z tile is double-buffered.
// Each CTA runs its own list of items (a tile and a range of terms) from a static schedule
// that balances the CTAs' costs (terms and cuts of Y_i).
// All waits are bounded; a wait that runs out raises the device status word.
#include "kpme_internal.cuh"

#include <algorithm>
#include "tc_common.cuh"

namespace kpme {
namespace {

using namespace tc;

constexpr int kBM = 128;
constexpr int kFBox = kBM * 128;        // 128 rows x 32 floats, 128-byte swizzle: 16 KB
constexpr int kTile = 2 * kFBox;        // 128 rows x 64 floats: 32 KB
constexpr int kACols = kSlices * 32;    // tensor-memory columns of one 64-wide A row's digits
constexpr int kA2Slice = kBM * 128;     // one digit plane of the Y_i tile in shared memory: 16 KB
constexpr int kBarBytes = 512;
constexpr int kThreads = 11 * 32;       // TMA, MMA, 4 converters, 4 epilogue warps, second MMA

struct OzfParams {
  int K, M, sb;
  const float* Y;      // stage-1 output: r0 planes of K^2 rows x K floats
  float* phi;
  const int2* pairs;   // (outer index, term)
  const int4* items;   // (m tile, first pair, end pair, 0)
  const int* cta;      // CTA c runs items [cta[c], cta[c + 1])
  int n_pairs, max_items;
  int* status;
  long long wait_cycles;   // budget of one bounded wait (clock cycles)
};

// float offset of (row, k) in a 128 x 64 float tile stored as two swizzled 128 x 32 boxes
__device__ __forceinline__ int tile_off(int row, int k) {
  return (k >> 5) * (kFBox / 4) + row * 32 + ((((k & 31) >> 2) ^ (row & 7)) << 2) + (k & 3);
}

// 4 floats (k = 4j .. 4j + 3) of one tile row
__device__ __forceinline__ float4 row_quad(const float* tile, int row, int j) {
  return *reinterpret_cast<const float4*>(tile + (j >> 3) * (kFBox / 4) + row * 32 + (((j & 7) ^ (row & 7)) << 2));
}

// Digits of one tile row into tensor memory columns taddr..: first the power of two above the
// row's maximum, then every group of 8 values gives four words of each digit plane (4 columns
// per plane).  The row is read from shared memory twice instead of being held in registers.
template <int K>
__device__ __forceinline__ void cut_row(const float* tile, int row, uint32_t taddr) {
  float m = 0.0f;
#pragma unroll
  for (int j = 0; j < K / 4; ++j) {
    const float4 x = row_quad(tile, row, j);
    m = fmaxf(m, fmaxf(fmaxf(fabsf(x.x), fabsf(x.y)), fmaxf(fabsf(x.z), fabsf(x.w))));
  }
  int e = 0;
  frexpf(m, &e);
  // kept rolled: the kernel's roles share the SM's instruction cache
#pragma unroll 1
  for (int g = 0; g < K / 8; ++g) {
    const float4 x0 = row_quad(tile, row, 2 * g), x1 = row_quad(tile, row, 2 * g + 1);
    const float v[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
    uint4 o[kSlices];
    slice8(v, e, o);
#pragma unroll
    for (int sl = 0; sl < kSlices; ++sl) tmem_st4(taddr + (uint32_t)(sl * 32 + 4 * g), o[sl]);
  }
}

// Digits of one Y_i row (held in registers: its K floats are loaded from global memory in one
// go, before the wait for the digit buffer) into the shared-memory A operand of step 2: four
// planes of 128 rows x 128 bytes (64 bf16), 16-byte chunks XOR-swizzled by row % 8, the
// K-major layout of the MMA's shared-memory descriptors (as TMA writes the factor tiles).
template <int K>
__device__ __forceinline__ void cut_row_smem(const float4 (&y)[K / 4], int r, uint8_t* a2s) {
  float m = 0.0f;
#pragma unroll
  for (int j = 0; j < K / 4; ++j)
    m = fmaxf(m, fmaxf(fmaxf(fabsf(y[j].x), fabsf(y[j].y)), fmaxf(fabsf(y[j].z), fabsf(y[j].w))));
  int e = 0;
  frexpf(m, &e);
  uint8_t* rb = a2s + (r >> 3) * 1024 + (r & 7) * 128;
#pragma unroll
  for (int g = 0; g < K / 8; ++g) {
    const float v[8] = {y[2 * g].x, y[2 * g].y, y[2 * g].z, y[2 * g].w,
                        y[2 * g + 1].x, y[2 * g + 1].y, y[2 * g + 1].z, y[2 * g + 1].w};
    uint4 o[kSlices];
    slice8(v, e, o);
#pragma unroll
    for (int sl = 0; sl < kSlices; ++sl) *reinterpret_cast<uint4*>(rb + sl * kA2Slice + ((g ^ (r & 7)) << 4)) = o[sl];
  }
}

template <int K>
__global__ void __launch_bounds__(kThreads, 1)
    mp_ozf_kernel(const __grid_constant__ CUtensorMap tmB2,
                  const __grid_constant__ CUtensorMap tmB1, OzfParams prm) {
  constexpr int BN = K;                 // both products have N = K
  constexpr int kBSlice = BN * 128;
  constexpr int kKSteps = K / 16;
  constexpr int kSub = kBM / K;         // k3' values per tile
  constexpr int kA3 = (512 - 4 * BN) / kACols >= 2 ? 2 : 1;   // Z_t digit slots after 2 accumulators
  static_assert(4 * BN + kA3 * kACols <= 512, "tensor memory layout");
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int bstage = kSlices * kBSlice;
  uint8_t* ring_b = smem;
  uint8_t* a2s = ring_b + prm.sb * bstage;                               // Y_i digits (A of step 2)
  float* ztile = reinterpret_cast<float*>(a2s + kSlices * kA2Slice);    // Z_t transposed, 2 buffers
  uint64_t* bars = reinterpret_cast<uint64_t*>(ztile + 2 * (kTile / 4));
  uint64_t* full_b = bars;
  uint64_t* empty_b = full_b + prm.sb;
  uint64_t* full_a2 = empty_b + prm.sb;
  uint64_t* empty_a2 = full_a2 + 1;
  uint64_t* d_full = empty_a2 + 1;     // [2] accumulators, taken by the ops in turn
  uint64_t* d_empty = d_full + 2;      // [2]
  uint64_t* full_z = d_empty + 2;      // [2]
  uint64_t* empty_z = full_z + 2;      // [2]
  uint64_t* full_a3 = empty_z + 2;     // [2] tensor-memory slots for Z_t digits
  uint64_t* empty_a3 = full_a3 + 2;    // [2]
  uint64_t* drain_bar = empty_a3 + 2;  // both MMA issuers' last commits, on the way out
  uint32_t* taddr_slot = reinterpret_cast<uint32_t*>(drain_bar + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(taddr_slot + 1);
  const WaitCtl wc{abort_flag, prm.status, prm.wait_cycles};
  int2* s_pairs = reinterpret_cast<int2*>(reinterpret_cast<uint8_t*>(bars) + kBarBytes);
  int4* s_items = reinterpret_cast<int4*>(s_pairs + ((prm.n_pairs + 1) & ~1));   // 16-byte aligned
  const int i_first = prm.cta[blockIdx.x];
  const int n_items = prm.cta[blockIdx.x + 1] - i_first;   // this CTA's items (<= max_items)
  for (int i = threadIdx.x; i < prm.n_pairs; i += blockDim.x) s_pairs[i] = prm.pairs[i];
  for (int i = threadIdx.x; i < n_items; i += blockDim.x) s_items[i] = prm.items[i_first + i];

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < prm.sb; ++s) {
      mbar_init(&full_b[s], 1);
      mbar_init(&empty_b[s], 2);   // the op's owner (commit) and the other MMA thread
    }
    mbar_init(full_a2, 4);
    mbar_init(empty_a2, 2);   // one commit from each MMA thread
    for (int b = 0; b < 2; ++b) {
      mbar_init(&d_full[b], 1);
      mbar_init(&d_empty[b], 4);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&full_z[b], 4);
      mbar_init(&empty_z[b], 4);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&full_a3[b], 4);
      mbar_init(&empty_a3[b], 2);  // the op's owner (commit) and the other MMA thread
    }
    mbar_init(drain_bar, 2);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(taddr_slot)),
                 "r"(512)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *taddr_slot;
  // tensor memory: two accumulators (ops in turn), kA3 slots of Z_t digits
  auto c_d = [](int b) { return (uint32_t)(b * 2 * BN); };
  auto c_a3 = [&](int slot) { return (uint32_t)(4 * BN + slot * kACols); };

  // The CTA's items form one stream of NT terms (items in order, each item's terms in order),
  // and the ops run over the stream, across item boundaries: S2(0), then S2(u), S3(u - 1) for
  // u = 1..NT-1, then S3(NT - 1); op o in [0, 2 NT): o = 0 -> S2(0), o = 2 NT - 1 -> S3(NT - 1),
  // else odd o -> S2((o+1)/2), even o -> S3(o/2 - 1).  Step 2 of an item's first term thus
  // runs while the previous item's last step 3 waits for its digits.
  auto op_of = [](int o, int n, bool& s2, int& j) {
    if (o == 0) {
      s2 = true;
      j = 0;
    } else if (o == 2 * n - 1) {
      s2 = false;
      j = n - 1;
    } else if (o & 1) {
      s2 = true;
      j = (o + 1) / 2;
    } else {
      s2 = false;
      j = o / 2 - 1;
    }
  };
  auto new_outer = [&](int p0, int j) { return j == 0 || s_pairs[p0 + j].x != s_pairs[p0 + j - 1].x; };
  // a cursor (item w, term j of the item) walks the stream in order
  struct Cur {
    int w, j;
  };
  auto n_of = [&](int w) { return s_items[w].z - s_items[w].y; };
  auto step = [&](Cur& c) {
    if (++c.j == n_of(c.w)) {
      ++c.w;
      c.j = 0;
    }
  };
  auto pidx = [&](const Cur& c) { return s_items[c.w].y + c.j; };
  auto c_newo = [&](const Cur& c) { return new_outer(s_items[c.w].y, c.j); };
  auto c_last_item = [&](const Cur& c) { return c.j + 1 == n_of(c.w); };
  // the next term of the stream needs a new cut of Y_i (its outer index or its tile changes)
  auto c_last_s2 = [&](const Cur& c) { return c_last_item(c) || new_outer(s_items[c.w].y, c.j + 1); };
  int NT = 0;
  for (int w = 0; w < n_items; ++w) NT += n_of(w);

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA: factor digits, in op order ----------------
      int ib = 0;
      bool ok = true;
      Cur c2{0, 0}, c3{0, 0};
      {
        for (int o = 0; o < 2 * NT && ok; ++o) {
          bool s2;
          int u;
          op_of(o, NT, s2, u);
          Cur& c = s2 ? c2 : c3;
          const int2 pr = s_pairs[pidx(c)];
          step(c);
          const int s = ib % prm.sb;
          if (ib >= prm.sb &&
              !mbar_wait(&empty_b[s], ((uint32_t)(ib / prm.sb) & 1u) ^ 1u, wc)) {
            ok = false;
            break;
          }
          uint8_t* dst = ring_b + s * bstage;
          mbar_expect_tx(&full_b[s], (uint32_t)(kSlices * kBSlice));
#pragma unroll
          for (int b = 0; b < kSlices; ++b)
            tma_load_3d(dst + b * kBSlice, s2 ? &tmB2 : &tmB1, &full_b[s], 0, pr.y * K, b);
          ++ib;
        }
      }
      drain_ring(full_b, prm.sb, ib, prm.status);   // loads in flight land before the CTA leaves
    }
  } else if (warp == 1 || warp == 10) {
    if (lane == 0) {
      // ---------------- MMA issue: two threads, one per accumulator ----------------
      // An issuing thread is held while the tensor pipe's queue is full, i.e. until its op is
      // nearly done, so one thread's waits for the next op would leave the pipe idle.  Thread
      // `mine` issues the ops of accumulator `mine` (every other op) and does its waits while
      // the other thread's op runs.  A parity wait is only unambiguous while the waiter is at
      // most one phase behind, so both threads walk the whole op sequence and wait for every
      // phase of the shared barriers (factor stages, Y_i and Z_t digits) in order, own op or
      // not, and those resources are released to their producers only when both threads have
      // passed them: the owner's commit (its MMAs done) plus the other thread's arrive.  The
      // Y_i digits are released right after the last step 2 that reads them, so the
      // converters cut the next Y_i while step 3 of the previous term runs.
      const int mine = warp == 1 ? 0 : 1;
      const uint32_t id = idesc_bf16(kBM, BN);
      int ib = 0, ia2 = 0, ja3 = 0, jd = 0;
      bool ok = true;
      // per stream term u (first 64): bit u of nmask = a new cut of Y_i starts at u, of lmask =
      // u is the last step 2 on its cut (read from shared memory once, not between MMAs)
      uint64_t nmask = 0, lmask = 0;
      if (NT <= 64) {
        Cur c{0, 0};
        for (int u = 0; u < NT; ++u) {
          nmask |= (uint64_t)c_newo(c) << u;
          lmask |= (uint64_t)c_last_s2(c) << u;
          step(c);
        }
      }
      Cur c2{0, 0};   // the next step 2's term (steps 3 need no term data here)
      {
        for (int o = 0; o < 2 * NT && ok; ++o) {
          bool s2;
          int u;
          op_of(o, NT, s2, u);
          bool newo_u = false, last_s2 = false;
          if (s2) {
            newo_u = NT <= 64 ? ((nmask >> u) & 1u) != 0 : c_newo(c2);
            last_s2 = NT <= 64 ? ((lmask >> u) & 1u) != 0 : c_last_s2(c2);
            step(c2);
          }
          const int slot = ja3 % kA3, db = jd & 1, s = ib % prm.sb;
          const bool own = db == mine;
          // the op's operands, observed by both threads in sequence order
          if (s2) {
            if (newo_u) {
              if (!mbar_wait(full_a2, (uint32_t)ia2 & 1u, wc)) {
                ok = false;
                break;
              }
              ++ia2;
            }
          } else if (!mbar_wait(&full_a3[slot], (uint32_t)(ja3 / kA3) & 1u, wc)) {
            ok = false;
            break;
          }
          if (!mbar_wait(&full_b[s], (uint32_t)(ib / prm.sb) & 1u, wc)) {
            ok = false;
            break;
          }
          if (!own) {   // the other thread's op: release what this thread has passed
            mbar_arrive(&empty_b[s]);
            if (!s2) mbar_arrive(&empty_a3[slot]);
            if (last_s2) mma_commit(empty_a2);   // this thread's earlier MMAs on the Y_i digits
            if (!s2) ++ja3;
            ++jd;
            ++ib;
            continue;
          }
          if (jd >= 2 && !mbar_wait(&d_empty[db], ((uint32_t)(jd >> 1) & 1u) ^ 1u, wc)) {
            ok = false;
            break;
          }
          fence_after();
          const uint32_t d = tmem + c_d(db);
          const uint64_t db0 = sdesc(smem_u32(ring_b + s * bstage));
          // the k steps in loops that are not unrolled (the ten products of a step are): the fully
          // unrolled issue code of both operand kinds stalled the issuing threads on instruction
          // fetch ("no instruction" 2.2 per issue; fused stages of the water box 103 -> 92 us)
          if (s2) {   // A: Y_i digits in shared memory
            const uint64_t da0 = sdesc(smem_u32(a2s));
#pragma unroll 1
            for (int kk = 0; kk < kKSteps; ++kk)
#pragma unroll
              for (int p = 0; p < kProducts; ++p) {
                const uint64_t dap = da0 + (uint64_t)((pa(p) * kA2Slice + kk * 32) >> 4);
                const uint64_t dbp = db0 + (uint64_t)((pb(p) * kBSlice + kk * 32) >> 4);
                const uint32_t acc = (kk == 0 && p <= 1) ? 0u : 1u;
                mma_bf16(p == 0 ? d : d + BN, dap, dbp, id, acc);
              }
          } else {    // A: Z_t digits in tensor memory
            const uint32_t a = tmem + c_a3(slot);
#pragma unroll 1
            for (int kk = 0; kk < kKSteps; ++kk)
#pragma unroll
              for (int p = 0; p < kProducts; ++p) {
                const uint32_t at = a + (uint32_t)(pa(p) * 32 + kk * 8);
                const uint64_t dbp = db0 + (uint64_t)((pb(p) * kBSlice + kk * 32) >> 4);
                const uint32_t acc = (kk == 0 && p <= 1) ? 0u : 1u;
                mma_bf16_ta(p == 0 ? d : d + BN, at, dbp, id, acc);
              }
          }
          mma_commit(&empty_b[s]);
          if (!s2) {
            mma_commit(&empty_a3[slot]);
            ++ja3;
          }
          if (last_s2) mma_commit(empty_a2);
          mma_commit(&d_full[db]);
          ++jd;
          ++ib;
        }
      }
      // every MMA issued by either thread has completed before tensor memory is released
      mma_commit(drain_bar);
      mbar_drain(drain_bar, 0, prm.status);
    }
  } else if (warp < 6) {
    // ---------- converters: digits of Y_i rows (shared memory) and of Z_t rows (tensor memory) ----------
    const int qd = warp & 3;
    const int r = 32 * qd + lane;
    const uint32_t lane_base = tmem + ((uint32_t)(32 * qd) << 16);
    const int64_t kk2 = (int64_t)K * K;
    int ia2 = 0, jz = 0, ja3 = 0;
    bool ok = true;
    Cur cy{0, 0};
    {
      // digits in the order the tensor pipe consumes them: Y_i of stream term t (when a new cut
      // starts there) before Z of term t - 1, since step 2 of term t precedes step 3 of t - 1
      for (int t = 0; t <= NT && ok; ++t) {
        const bool cut_y = t < NT && c_newo(cy);
        const int m0 = t < NT ? s_items[cy.w].x * kBM : 0;
        const int outer = t < NT ? s_pairs[pidx(cy)].x : 0;
        if (t < NT) step(cy);
        if (cut_y) {
          // the row's loads are in flight while this warp waits for the digit buffer
          const float4* y4 = reinterpret_cast<const float4*>(prm.Y + ((int64_t)outer * kk2 + m0 + r) * K);
          float4 y[K / 4];
#pragma unroll
          for (int q = 0; q < K / 4; ++q) y[q] = __ldg(y4 + q);
          if (ia2 >= 1 &&
              !__all_sync(0xffffffffu, mbar_wait(empty_a2, ((uint32_t)ia2 & 1u) ^ 1u, wc))) {
            ok = false;
            break;
          }
          cut_row_smem<K>(y, r, a2s);
          // generic-proxy writes, read by the tensor pipe (async proxy)
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          mbar_arrive_warp(full_a2);
          ++ia2;
        }
        if (t == 0) continue;
        const int zb = jz & 1, slot = ja3 % kA3;
        if (!__all_sync(0xffffffffu, mbar_wait(&full_z[zb], (uint32_t)(jz >> 1) & 1u, wc)) ||
            (ja3 >= kA3 && !__all_sync(0xffffffffu, mbar_wait(&empty_a3[slot], ((uint32_t)(ja3 / kA3) & 1u) ^ 1u,
                                                              wc)))) {
          ok = false;
          break;
        }
        fence_after();
        cut_row<K>(ztile + zb * (kTile / 4), r, lane_base + c_a3(slot));
        mbar_arrive_warp(&empty_z[zb]);
        ++jz;
        tmem_wait_st();
        fence_before();
        mbar_arrive_warp(&full_a3[slot]);
        ++ja3;
      }
    }
    tmem_wait_st();
  } else {
    // ---------------- epilogue, in the MMA's op order ----------------
    // step 2 of term j: Z_t = D0 + D1 written transposed (thread = tile row m = (k3' = m / K,
    // k1 = m % K); Z_t(m, k2') to row k3' K + k2', column k1);
    // step 3 of term j: the Phi tile rows rho = (k3' = rho / K, k2' = rho % K), columns k1',
    // summed over the item's terms in registers and added atomically at the item's end.
    const int qd = warp & 3;
    const int m = 32 * qd + lane;
    const int sub = m / K, k1 = m % K;
    const uint32_t lane_base = tmem + ((uint32_t)(32 * qd) << 16);
    // float offsets of (row sub K + c, column k1) in a Z tile: c * 32 + zoff[c % 8]
    // (the 16-byte chunk index is XORed with row % 8 = c % 8, since K % 8 == 0)
    int zoff[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) zoff[c] = tile_off(sub * K + c, k1) - c * 32;
    int jd = 0, jz = 0;
    bool ok = true;
    Cur c3{0, 0};   // the next step 3's term
    float acc[BN];
#pragma unroll
    for (int c = 0; c < BN; ++c) acc[c] = 0.0f;
    {
      for (int o = 0; o < 2 * NT; ++o) {
        bool s2;
        int u;
        op_of(o, NT, s2, u);
        if (!ok) continue;
        const int zb = jz & 1;
        if ((s2 && jz >= 2 &&
             !__all_sync(0xffffffffu, mbar_wait(&empty_z[zb], ((uint32_t)(jz >> 1) & 1u) ^ 1u, wc))) ||
            !__all_sync(0xffffffffu, mbar_wait(&d_full[jd & 1], (uint32_t)(jd >> 1) & 1u, wc))) {
          ok = false;
          continue;
        }
        fence_after();
        const uint32_t dcol = lane_base + c_d(jd & 1);
        if (s2) {
          float* zt = ztile + zb * (kTile / 4);
#pragma unroll 1
          for (int c0 = 0; c0 < BN; c0 += 16) {
            uint32_t a0[16], a1[16];
            tmem_ld16(dcol + (uint32_t)c0, a0);
            tmem_ld16(dcol + (uint32_t)(BN + c0), a1);
            tmem_wait_ld();
            float* zc = zt + c0 * 32;
#pragma unroll
            for (int i = 0; i < 16; ++i) zc[i * 32 + zoff[i & 7]] = __uint_as_float(a0[i]) + __uint_as_float(a1[i]);
          }
        } else {
#pragma unroll
          for (int c0 = 0; c0 < BN; c0 += 16) {
            uint32_t a0[16], a1[16];
            tmem_ld16(dcol + (uint32_t)c0, a0);
            tmem_ld16(dcol + (uint32_t)(BN + c0), a1);
            tmem_wait_ld();
#pragma unroll
            for (int i = 0; i < 16; ++i) acc[c0 + i] += __uint_as_float(a0[i]) + __uint_as_float(a1[i]);
          }
        }
        fence_before();
        mbar_arrive_warp(&d_empty[jd & 1]);
        ++jd;
        if (s2) {
          mbar_arrive_warp(&full_z[zb]);
          ++jz;
          continue;
        }
        // step 3: at the last term of an item its Phi tile is complete
        const bool flush = c_last_item(c3);
        const int m0 = s_items[c3.w].x * kBM;
        step(c3);
        if (!flush || *abort_flag) continue;
        // Phi[k1'][k2'][k3'] for this thread's row rho = m: k3' = m0 / K + m / K, k2' = m % K
        const int k3 = m0 / K + sub, k2 = k1;
        float* out = prm.phi + (int64_t)k2 * K + k3;
#pragma unroll
        for (int c = 0; c < BN; ++c) {
          atomicAdd(out + (int64_t)c * K * K, acc[c]);
          acc[c] = 0.0f;
        }
      }
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 1) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
  }
  (void)kSub;
}

template <int K>
cudaError_t launch_k(kpme_plan_t P, const OzfArgs& a, OzfParams prm) {
  const int bstage = kSlices * K * 128;
  prm.sb = (K == 64) ? 3 : 6;
  const int fixed = kSlices * kA2Slice + 2 * kTile + kBarBytes + ((prm.n_pairs + 1) & ~1) * (int)sizeof(int2) +
                    prm.max_items * (int)sizeof(int4) + 1024;
  while (prm.sb > 2 && prm.sb * bstage + fixed > 227 * 1024) --prm.sb;   // long pair tables
  const int smem = prm.sb * bstage + fixed;
  if (smem > 227 * 1024) return cudaErrorInvalidValue;
  auto kern = mp_ozf_kernel<K>;
  cudaError_t e = raise_smem_cap(reinterpret_cast<const void*>(kern));
  if (e != cudaSuccess) return e;
  const dim3 grid((unsigned)a.jobs->h_cta.size() - 1);   // one CTA per range of the static schedule
  kern<<<grid, kThreads, smem, P->stream>>>(*a.tmB2, *a.tmB1, prm);
  return cudaGetLastError();
}

}  // namespace

bool ozf_supported(int K) { return K == 32 || K == 64; }

cudaError_t launch_mp_ozf(kpme_plan_t P, const OzfArgs& a) {
  OzfParams prm{};
  prm.K = a.K;
  prm.M = a.K * a.K;
  prm.phi = a.phi;
  prm.Y = a.Y;
  if (a.jobs->h_cta.size() < 2 || !a.jobs->d_items || !a.jobs->d_cta) return cudaErrorInvalidValue;
  prm.pairs = a.jobs->d_pairs;
  prm.items = a.jobs->d_items;
  prm.cta = a.jobs->d_cta;
  prm.n_pairs = (int)a.jobs->h_pairs.size();
  prm.max_items = 0;
  for (size_t c = 0; c + 1 < a.jobs->h_cta.size(); ++c)
    prm.max_items = std::max(prm.max_items, a.jobs->h_cta[c + 1] - a.jobs->h_cta[c]);
  prm.status = P->d_status;
  prm.wait_cycles = P->wait_cycles;
  if (a.K == 64) return launch_k<64>(P, a, prm);
  if (a.K == 32) return launch_k<32>(P, a, prm);
  return cudaErrorInvalidValue;
}

}  // namespace kpme
