// Error-free split mode products with the A operand in tensor memory (KPME_BF16X10, K % 16 == 0, K >= 32).
//
// Same contraction and arithmetic as gemm_oz.cu (each operand row cut into four fixed-point
// bf16 digits relative to a common power of two, ten digit products per multiply, the leading
// one into an exactly accumulated D0 and the nine others into D1; Ozaki, Ogita, Oishi and Rump,
// Numer. Algorithms 59, 2012), with a different data path for A:
//   * float32 A rows (the charge mesh Q, Y_i or Z_t) come into shared memory by TMA, two
//     128-row x 32-float boxes per 64-wide k chunk (128-byte swizzle), and converter warps cut
//     them into digits with the row's power of two and store the digits straight into tensor
//     memory (tcgen05.st, one row per TMEM lane).  The MMAs read A from tensor memory and only
//     the factor digits from shared memory, so an N = 64 MMA is not bound by shared-memory
//     reads, and the factor ring can be deep;
//   * A_RES: every pair of an item shares one A tile (stage 1: Q for several outer factors;
//     stage 2: Y_i for several terms of outer term i), cut once per item and kept in tensor
//     memory while its pairs run; every pair stores its own output plane and publishes the
//     next stage's row maxima (mode 2);
//   * otherwise (stage 3) every pair has its own A (Z_t), cut per 64-wide chunk into a ring of
//     two tensor-memory slots, and the item's pairs are summed (mode 1, float32 atomics).
// Folded factors (fold): every factor is a real symmetric circulant, so it commutes with the
// reflection a <-> K - 1 - a of its axis, which has no fixed point for even K; in the basis of
// sums x(a) + x(K-1-a) and differences x(a) - x(K-1-a) it is block diagonal with two K/2 x K/2
// blocks.  With the mesh in that basis on all three axes, an item whose output columns lie in
// one half contracts only the K/2 values of that half: half the digit products of every stage.
// All waits are bounded; a wait that runs out raises the device status word and every role
// drains without further waits.
#include "kpme_internal.cuh"
#include "tc_common.cuh"
#include "df.cuh"

#include <algorithm>

namespace kpme {
namespace {

using namespace tc;

constexpr int kBM = 128;
constexpr int kChunk = 64;
constexpr int kFBox = kBM * 128;                      // one 128-row x 32-float box: 16 KB
constexpr int kFStage = 2 * kFBox;                    // float32 staging of one chunk: 32 KB
constexpr int kChunkCols = kSlices * kChunk / 2;      // TMEM columns of one chunk's four digit planes
constexpr int kBarBytes = 512;

struct OztParams {
  int M, N, Kr, kchunks;
  int kc;               // contracted values per item: Kr, or Kr / 2 with folded factors
  int fold;             // folded: items of output columns n >= Kr / 2 read A columns [Kr/2, Kr)
  int self_max;         // the converters take each row's power of two from the staged chunks of
                        // the row (every chunk of a unit staged at once, one thread per row);
                        // rowmax_in is not read
  int tile_max;         // mode 2: rowmax_out receives one max |value| per (plane, item tile);
                        // A per pair: rowmax_in holds those maxima and a row takes the one of
                        // the tile its half-row was written in (K = 2 kBM, BN = 128, fold)
  int sb, bstage;       // factor ring: stages and bytes per stage
  int sf;               // float32 staging stages
  int nacc, nat;        // accumulator buffers (2 BN columns each); A slots
  int a_col0, at_cols;  // first A column; columns per A slot
  int mode;             // 1: sum the item's pairs into out (atomics); 2: store each pair
  const float* rowmax_in;
  int64_t rm_in_bs;
  float* out;
  int64_t out_bs;
  int out_base;         // mode 2: pair (a, f) writes plane f - out_base
  float* rowmax_out;
  int64_t rm_out_bs;
  const int* start;
  const int2* pairs;
  int n_jobs, n_pairs;
  int* status;
  long long wait_cycles;   // budget of one bounded wait (clock cycles)
};

template <int NCONV>
constexpr int ozt_threads() { return 64 + 32 * NCONV + 128; }

// warp 0: TMA (float32 A boxes and factor digits); warp 1: TMEM allocation and MMA issue;
// warps 2 .. NCONV + 1: converters (TMEM lane quadrant warp % 4, k half (warp - 2) / 4 when
// NCONV = 8); last four warps: epilogue (lane quadrant warp % 4).
template <int BN, int NCONV, bool A_RES>
__global__ void __launch_bounds__(ozt_threads<NCONV>(), 1)
    mp_ozt_kernel(const __grid_constant__ CUtensorMap tmF, const __grid_constant__ CUtensorMap tmB, OztParams prm) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  constexpr int kBSlice = BN * 128;
  constexpr int kParts = NCONV / 4;                 // converter threads per row
  constexpr int kHalves = 2 / kParts;               // 32-wide k halves per converter thread and chunk
  uint8_t* ring_b = smem;
  uint8_t* ring_f = smem + prm.sb * prm.bstage;
  uint64_t* full_b = reinterpret_cast<uint64_t*>(ring_f + prm.sf * kFStage);
  uint64_t* empty_b = full_b + prm.sb;
  uint64_t* full_f = empty_b + prm.sb;
  uint64_t* empty_f = full_f + prm.sf;
  uint64_t* full_t = empty_f + prm.sf;
  uint64_t* empty_t = full_t + prm.nat;
  uint64_t* acc_full = empty_t + prm.nat;
  uint64_t* acc_empty = acc_full + prm.nacc;
  uint64_t* drain_bar = acc_empty + prm.nacc;   // the MMA issuer's last commit, on the way out
  uint32_t* taddr_slot = reinterpret_cast<uint32_t*>(drain_bar + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(taddr_slot + 1);
  const WaitCtl wc{abort_flag, prm.status, prm.wait_cycles};
  unsigned int* red = reinterpret_cast<unsigned int*>(reinterpret_cast<uint8_t*>(full_b) + kBarBytes);
  // the job tables live in shared memory: every role reads them for every item and pair
  int2* s_pairs = reinterpret_cast<int2*>(red + 4 * BN);
  int* s_start = reinterpret_cast<int*>(s_pairs + prm.n_pairs);
  for (int i = threadIdx.x; i < prm.n_pairs; i += blockDim.x) s_pairs[i] = prm.pairs[i];
  for (int i = threadIdx.x; i <= prm.n_jobs; i += blockDim.x) s_start[i] = prm.start[i];

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m_tiles = (prm.M + kBM - 1) / kBM;
  const int n_tiles = prm.N / BN;
  const int n_items = m_tiles * n_tiles * prm.n_jobs;
  const int kchunks = prm.kchunks;
  constexpr int kEpi0 = 2 + NCONV;

  if (threadIdx.x == 0) {
    for (int s = 0; s < prm.sb; ++s) {
      mbar_init(&full_b[s], 1);
      mbar_init(&empty_b[s], 1);
    }
    for (int s = 0; s < prm.sf; ++s) {
      mbar_init(&full_f[s], 1);
      mbar_init(&empty_f[s], 32 * NCONV);
    }
    for (int s = 0; s < prm.nat; ++s) {
      mbar_init(&full_t[s], 32 * NCONV);
      mbar_init(&empty_t[s], 1);
    }
    for (int b = 0; b < prm.nacc; ++b) {
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
                 "r"(512)
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
  // boxes of chunk c that hold valid k (the second is skipped when it starts at or past kc)
  auto boxes = [&](int c) { return (c * kChunk + 32 < prm.kc) ? 2 : 1; };
  // first A column of an item: its output half's block on folded factors
  auto a_k0 = [&](int n0) { return (prm.fold && n0 >= prm.Kr / 2) ? prm.Kr / 2 : 0; };

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA: float32 A boxes and factor digits ----------------
      int jf = 0, ib = 0;
      bool ok = true;
      auto load_f = [&](int plane, int m0, int k0, int c) -> bool {
        const int s = jf % prm.sf;
        const uint32_t ph = (uint32_t)(jf / prm.sf) & 1u;
        if (jf >= prm.sf && !mbar_wait(&empty_f[s], ph ^ 1u, wc)) return false;
        uint8_t* dst = ring_f + s * kFStage;
        const int nb = boxes(c);
        mbar_expect_tx(&full_f[s], (uint32_t)(nb * kFBox));
        for (int b = 0; b < nb; ++b)
          tma_load_3d(dst + b * kFBox, &tmF, &full_f[s], k0 + c * kChunk + 32 * b, m0, plane);
        ++jf;
        return true;
      };
      auto load_b = [&](int fac, int n0, int c) -> bool {
        const int s = ib % prm.sb;
        const uint32_t ph = (uint32_t)(ib / prm.sb) & 1u;
        if (ib >= prm.sb && !mbar_wait(&empty_b[s], ph ^ 1u, wc)) return false;
        uint8_t* dst = ring_b + s * prm.bstage;
        mbar_expect_tx(&full_b[s], (uint32_t)(kSlices * kBSlice));
#pragma unroll
        for (int b = 0; b < kSlices; ++b)
          tma_load_3d(dst + b * kBSlice, &tmB, &full_b[s], c * kChunk, fac * prm.N + n0, b);
        ++ib;
        return true;
      };
      for (int w = blockIdx.x; w < n_items && ok; w += gridDim.x) {
        int m0, n0, job;
        decode(w, m0, n0, job);
        const int p0 = s_start[job], p1 = s_start[job + 1];
        const int k0 = a_k0(n0);
        if constexpr (A_RES) {
          const int plane = s_pairs[p0].x;
          for (int c = 0; c < kchunks && ok; ++c) ok = load_f(plane, m0, k0, c);
        }
        for (int p = p0; p < p1 && ok; ++p) {
          const int2 pr = s_pairs[p];
          for (int c = 0; c < kchunks && ok; ++c) {
            if constexpr (!A_RES) ok = load_f(pr.x, m0, k0, c);
            if (ok) ok = load_b(pr.y, n0, c);
          }
        }
      }
      // loads in flight land before the CTA leaves (at once unless a wait gave up)
      drain_ring(full_f, prm.sf, jf, prm.status);
      drain_ring(full_b, prm.sb, ib, prm.status);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issue ----------------
      const uint32_t id = idesc_bf16(kBM, BN);
      int ib = 0, it = 0, pc = 0;
      bool ok = true;
      for (int w = blockIdx.x; w < n_items && ok; w += gridDim.x) {
        int m0, n0, job;
        decode(w, m0, n0, job);
        const int np = s_start[job + 1] - s_start[job];
        int slot = 0;
        uint32_t a_item = 0;
        if constexpr (A_RES) {
          slot = it % prm.nat;
          if (!mbar_wait(&full_t[slot], (uint32_t)(it / prm.nat) & 1u, wc)) break;
          fence_after();
          a_item = tmem + (uint32_t)(prm.a_col0 + slot * prm.at_cols);
        }
        for (int pl = 0; pl < np && ok; ++pl, ++pc) {
          const int buf = pc % prm.nacc;
          if (pc >= prm.nacc &&
              !mbar_wait(&acc_empty[buf], (uint32_t)((pc / prm.nacc) - 1) & 1u, wc)) {
            ok = false;
            break;
          }
          fence_after();
          const uint32_t d0 = tmem + (uint32_t)(buf * 2 * BN), d1 = d0 + BN;
          for (int c = 0; c < kchunks; ++c) {
            uint32_t a_c;
            if constexpr (A_RES) {
              a_c = a_item + (uint32_t)(c * kChunkCols);
            } else {
              slot = it % prm.nat;
              if (!mbar_wait(&full_t[slot], (uint32_t)(it / prm.nat) & 1u, wc)) {
                ok = false;
                break;
              }
              a_c = tmem + (uint32_t)(prm.a_col0 + slot * prm.at_cols);
            }
            const int s = ib % prm.sb;
            if (!mbar_wait(&full_b[s], (uint32_t)(ib / prm.sb) & 1u, wc)) {
              ok = false;
              break;
            }
            fence_after();
            int ksteps = (prm.kc - c * kChunk + 15) / 16;
            ksteps = ksteps > 4 ? 4 : ksteps;
            // one descriptor per stage; the digit planes and k steps are compile-time offsets
            // added to its 14-bit address field (addresses stay below 256 KB: no carry)
            const uint64_t db0 = sdesc(smem_u32(ring_b + s * prm.bstage));
            auto kstep = [&](int kk, bool first) {
#pragma unroll
              for (int p = 0; p < kProducts; ++p) {
                const uint32_t at = a_c + (uint32_t)(pa(p) * (kChunk / 2) + kk * 8);
                const uint64_t db = db0 + (uint64_t)((pb(p) * kBSlice + kk * 32) >> 4);
                if (p == 0)
                  mma_bf16_ta(d0, at, db, id, first ? 0u : 1u);
                else
                  mma_bf16_ta(d1, at, db, id, (first && p == 1) ? 0u : 1u);
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
            mma_commit(&empty_b[s]);
            ++ib;
            if constexpr (!A_RES) {
              mma_commit(&empty_t[slot]);
              ++it;
            }
          }
          if (!ok) break;
          mma_commit(&acc_full[buf]);
        }
        if constexpr (A_RES) {
          if (!ok) break;
          mma_commit(&empty_t[slot]);
          ++it;
        }
      }
      // every MMA issued has completed before tensor memory is released
      mma_commit(drain_bar);
      mbar_drain(drain_bar, 0, prm.status);
    }
  } else if (warp < kEpi0) {
    // ---------------- converters: float32 rows -> digits in tensor memory ----------------
    const int qd = warp & 3;
    const int r = 32 * qd + lane;                         // tile row = TMEM lane
    const int h_first = kParts == 2 ? (warp - 2) / 4 : 0;  // first 32-wide k half of this thread
    const uint32_t lane_base = tmem + ((uint32_t)(32 * qd) << 16);
    int jf = 0, it = 0;
    bool ok = true;
    for (int w = blockIdx.x; w < n_items && ok; w += gridDim.x) {
      int m0, n0, job;
      decode(w, m0, n0, job);
      const int row = m0 + r;
      const bool valid = row < prm.M;
      const int p0 = s_start[job], p1 = s_start[job + 1];
      const int nunits = A_RES ? 1 : p1 - p0;
      // entry of this row in the unit's maxima: the row itself, or (tile_max) the stage-2 tile
      // holding its half-row: row = n (M / Kr) + g is column n of the rows g Kr + [k0, k0 + kc)
      int64_t rm_entry = row;
      if (prm.tile_max) {
        const int rows_per_col = prm.M / prm.Kr;
        const int n = row / rows_per_col, g = row - n * rows_per_col;
        rm_entry = (int64_t)((g * prm.Kr + a_k0(n0)) / kBM) * (prm.Kr / BN) + n / BN;
      }
      // the row maximum of unit u + 1 is loaded while unit u is cut
      float rm_next = (valid && !prm.self_max) ? prm.rowmax_in[(int64_t)s_pairs[p0].x * prm.rm_in_bs + rm_entry] : 0.0f;
      for (int u = 0; u < nunits && ok; ++u) {
        float rm = rm_next;
        if (u + 1 < nunits && !prm.self_max)
          rm_next = valid ? prm.rowmax_in[(int64_t)s_pairs[p0 + u + 1].x * prm.rm_in_bs + rm_entry] : 0.0f;
        if (prm.self_max) {
          // every chunk of this unit is staged at once (kchunks <= sf): the maximum of the
          // thread's row over the unit's k range, read from the staging buffers, which stay
          // held until each chunk is cut below (their phases are waited again there at once)
          rm = 0.0f;
          for (int c = 0; c < kchunks && ok; ++c) {
            const int jc = jf + c, s = jc % prm.sf;
            if (!__all_sync(0xffffffffu, mbar_wait(&full_f[s], (uint32_t)(jc / prm.sf) & 1u, wc))) {
              ok = false;
              break;
            }
            const uint8_t* stg = ring_f + s * kFStage;
#pragma unroll
            for (int hh = 0; hh < kHalves; ++hh) {
              const uint8_t* rowp = stg + (h_first + hh) * kFBox + r * 128;
#pragma unroll
              for (int j = 0; j < 8; ++j) {
                const float4 x = *reinterpret_cast<const float4*>(rowp + ((j ^ (r & 7)) << 4));
                rm = fmaxf(rm, fmaxf(fmaxf(fabsf(x.x), fabsf(x.y)), fmaxf(fabsf(x.z), fabsf(x.w))));
              }
            }
          }
          if (!ok) break;
        }
        int e = 0;
        frexpf(rm, &e);
        int slot = 0;
        uint32_t col_unit = 0;
        if constexpr (A_RES) {
          slot = it % prm.nat;
          if (it >= prm.nat &&
              !__all_sync(0xffffffffu, mbar_wait(&empty_t[slot], ((uint32_t)(it / prm.nat) & 1u) ^ 1u, wc))) {
            ok = false;
            break;
          }
          fence_after();
          col_unit = (uint32_t)(prm.a_col0 + slot * prm.at_cols);
        }
        for (int c = 0; c < kchunks; ++c) {
          const int s = jf % prm.sf;
          if (!__all_sync(0xffffffffu,
                          mbar_wait(&full_f[s], (uint32_t)(jf / prm.sf) & 1u, wc))) {
            ok = false;
            break;
          }
          uint32_t col;
          if constexpr (A_RES) {
            col = col_unit + (uint32_t)(c * kChunkCols);
          } else {
            slot = it % prm.nat;
            if (it >= prm.nat &&
                !__all_sync(0xffffffffu, mbar_wait(&empty_t[slot], ((uint32_t)(it / prm.nat) & 1u) ^ 1u,
                                                   wc))) {
              ok = false;
              break;
            }
            fence_after();
            col = (uint32_t)(prm.a_col0 + slot * prm.at_cols);
          }
          // the thread's 32-wide k halves and their groups of 8 values one at a time, in loops
          // that are not unrolled: the unrolled cut of a whole chunk made the converters' code so
          // long that instruction fetch stalled the warps sharing their SM sub-partitions, the
          // MMA issuer among them (stage 3 of the 10^6-charge box: 6.44 -> 5.23 ms with the
          // halves rolled, -> 5.08 ms with the groups too)
          const uint8_t* stg = ring_f + s * kFStage;
#pragma unroll 1
          for (int hh = 0; hh < kHalves; ++hh) {
            const int h = h_first + hh;
            if (c * kChunk + 32 * h >= prm.kc) continue;   // warp-uniform: k half past the end
            const uint8_t* rowp = stg + h * kFBox + r * 128;
#pragma unroll 1
            for (int g = 0; g < 4; ++g) {
              const float4 x0 = *reinterpret_cast<const float4*>(rowp + (((2 * g) ^ (r & 7)) << 4));
              const float4 x1 = *reinterpret_cast<const float4*>(rowp + (((2 * g + 1) ^ (r & 7)) << 4));
              const float v[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
              uint4 o[kSlices];
              slice8(v, e, o);
#pragma unroll
              for (int sl = 0; sl < kSlices; ++sl)
                tmem_st4(lane_base + col + (uint32_t)(sl * (kChunk / 2) + 16 * h + 4 * g), o[sl]);
            }
          }
          mbar_arrive(&empty_f[s]);
          ++jf;
          if constexpr (!A_RES) {
            tmem_wait_st();
            fence_before();
            mbar_arrive(&full_t[slot]);
            ++it;
          }
        }
        if constexpr (A_RES) {
          if (!ok) break;
          tmem_wait_st();
          fence_before();
          mbar_arrive(&full_t[slot]);
          ++it;
        }
      }
    }
    tmem_wait_st();   // a unit given up half cut: its stores complete before the release
  } else {
    // ---------------- epilogue ----------------
    // Every epilogue thread runs every item and every pair, and (mode 2) the same number of
    // named-barrier syncs, whatever happens to its waits (a failed wait only skips work).
    const int wq = warp & 3;
    const int r = 32 * wq + lane;
    const uint32_t lane_base = tmem + ((uint32_t)(32 * wq) << 16);
    int pc = 0;
    bool ok = true;
    for (int w = blockIdx.x; w < n_items; w += gridDim.x) {
      int m0, n0, job;
      decode(w, m0, n0, job);
      const int row = m0 + r;
      const int p0 = s_start[job];
      const int np = s_start[job + 1] - p0;
      float acc[BN];
#pragma unroll
      for (int c = 0; c < BN; ++c) acc[c] = 0.0f;
      for (int pl = 0; pl < np; ++pl, ++pc) {
        if (prm.mode == 2) {
#pragma unroll
          for (int c = 0; c < BN; ++c) acc[c] = 0.0f;
        }
        if (ok) {
          const int buf = pc % prm.nacc;
          const bool got = __all_sync(0xffffffffu, mbar_wait(&acc_full[buf], (uint32_t)(pc / prm.nacc) & 1u,
                                                             wc));
          if (!got) {
            ok = false;
          } else {
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
        }
        if (prm.mode != 2) continue;
        // ---- mode 2: this pair's output plane and the next stage's row maxima ----
        const bool live = ok && !*abort_flag && row < prm.M;
        const int plane = s_pairs[p0 + pl].y - prm.out_base;
        if (live) {
          float* o = prm.out + (int64_t)plane * prm.out_bs + (int64_t)n0 * prm.M + row;
#pragma unroll
          for (int c = 0; c < BN; ++c) o[(int64_t)c * prm.M] = acc[c];
        }
        if (prm.rowmax_out == nullptr) continue;
        if (prm.tile_max) {
          // one max |value| of this pair's 128 x BN tile (a plain store: each tile is written
          // by one pair), for the power of two of the next stage's rows that read it
          float tm = 0.0f;
#pragma unroll
          for (int c = 0; c < BN; ++c) tm = fmaxf(tm, fabsf(acc[c]));
          const unsigned int wm = __reduce_max_sync(0xffffffffu, live ? __float_as_uint(tm) : 0u);
          if (lane == 0) red[wq] = wm;
          asm volatile("bar.sync 1, 128;" ::: "memory");
          if (wq == 0 && lane == 0 && live)
            prm.rowmax_out[(int64_t)plane * prm.rm_out_bs + (int64_t)(m0 / kBM) * n_tiles + n0 / BN] =
                __uint_as_float(max(max(red[0], red[1]), max(red[2], red[3])));
          asm volatile("bar.sync 1, 128;" ::: "memory");
          continue;
        }
        // the consuming row (n, row / K) spans K consecutive rows of column n
        const int K = prm.Kr;
        const int64_t rows_next = prm.M / K;
        unsigned int* dst = reinterpret_cast<unsigned int*>(prm.rowmax_out + (int64_t)plane * prm.rm_out_bs) +
                            (int64_t)n0 * rows_next;
        constexpr int kJ = (BN + 31) / 32;
        if (K % 32 != 0) {
          // (K % 32 != 0, K > 32) a warp's 32 rows reach at most two consuming rows g_w and
          // g_w + 1: the warp's maximum of each part, one atomic per column and part (the same
          // branch for every epilogue thread: no named barrier here)
          const int gw = (m0 + 32 * wq) / K;
          const bool upper = row / K != gw;
          unsigned int lo[kJ], hi[kJ];
#pragma unroll
          for (int j = 0; j < kJ; ++j) lo[j] = hi[j] = 0u;
#pragma unroll
          for (int c = 0; c < BN; ++c) {
            const unsigned int b = live ? __float_as_uint(fabsf(acc[c])) : 0u;
            const unsigned int ml = __reduce_max_sync(0xffffffffu, upper ? 0u : b);
            const unsigned int mh = __reduce_max_sync(0xffffffffu, upper ? b : 0u);
            if ((c & 31) == lane) {
              lo[c >> 5] = ml;
              hi[c >> 5] = mh;
            }
          }
#pragma unroll
          for (int j = 0; j < kJ; ++j) {
            const int c = 32 * j + lane;
            if (c >= BN) continue;
            if (lo[j] != 0u) atomicMax(dst + (int64_t)c * rows_next + gw, lo[j]);
            if (hi[j] != 0u) atomicMax(dst + (int64_t)c * rows_next + gw + 1, hi[j]);
          }
          continue;
        }
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
      }
      if (prm.mode == 1 && ok && !*abort_flag && row < prm.M) {
        float* o = prm.out + (int64_t)n0 * prm.M + row;
#pragma unroll
        for (int c = 0; c < BN; ++c) atomicAdd(o + (int64_t)c * prm.M, acc[c]);
      }
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 1) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
  }
}

// Row maxima of a float32 tensor of rows x K values (one warp per row): max |x| per row.
// Optionally zeroes nz floats of `zero` (the potential mesh the following stages accumulate
// into), which saves a separate clearing node on the path.
__global__ void rowmax_rows_kernel(const float* __restrict__ in, int64_t rows, int K, float* __restrict__ out,
                                   float* __restrict__ zero, int64_t nz) {
  if (zero)
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nz; i += (int64_t)gridDim.x * blockDim.x)
      zero[i] = 0.0f;
  const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= rows) return;
  const float* row = in + w * K;
  float m = 0.0f;
  for (int k = lane; k < K; k += 32) m = fmaxf(m, fabsf(row[k]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (lane == 0) out[w] = m;
}

struct OztConfig {
  int sb, sf, nacc, nat, a_col0, at_cols, smem;
};

OztConfig ozt_config(int bn, int K, bool a_res) {
  OztConfig c{};
  const int kchunks = (K + kChunk - 1) / kChunk;
  const int bstage = kSlices * bn * 128;
  // A per pair (stage 3) streams a new float32 A for every pair from DRAM: three staging
  // buffers keep more of it in flight where the factor ring keeps three stages; A resident
  // across an item's pairs needs two
  c.sf = (!a_res && (200 * 1024 - 3 * kFStage) / bstage >= 3) ? 3 : 2;
  c.sb = (200 * 1024 - c.sf * kFStage) / bstage;
  if (c.sb > 8) c.sb = 8;
  const int acc_cols = 2 * bn;
  // tensor memory: two accumulators (the epilogue drains one while the MMAs fill the other)
  // when A fits beside them, else one (BN = 128: the N = 128 MMAs halve the instructions per
  // flop, and the epilogue's drain of the single accumulator is short against a pair's MMAs)
  c.at_cols = a_res ? kchunks * kChunkCols : kChunkCols;
  const int want_nat = a_res ? 1 : 2;
  c.nacc = (512 - want_nat * c.at_cols) / acc_cols;
  if (c.nacc > 4) c.nacc = 4;
  c.nat = c.nacc > 0 ? (512 - c.nacc * acc_cols) / c.at_cols : 0;
  if (c.nat > 2) c.nat = 2;
  c.a_col0 = c.nacc * acc_cols;
  c.smem = c.sb * bstage + c.sf * kFStage + kBarBytes + 4 * bn * 4 + 1024;
  return c;
}

template <int BN, int NCONV, bool A_RES>
cudaError_t launch_cfg(cudaStream_t st, const CUtensorMap* tmF, const CUtensorMap* tmB, const OztParams& prm,
                       dim3 grid, int smem) {
  auto kern = mp_ozt_kernel<BN, NCONV, A_RES>;
  cudaError_t e = raise_smem_cap(reinterpret_cast<const void*>(kern));
  if (e != cudaSuccess) return e;
  kern<<<grid, ozt_threads<NCONV>(), smem, st>>>(*tmF, *tmB, prm);
  return cudaGetLastError();
}

template <int BN>
cudaError_t launch_bn(const OztArgs& a, cudaStream_t st, const OztParams& prm, dim3 grid, int smem) {
  // BN = 128: four converter warps (one full 64-wide row per thread), so that the epilogue's
  // 128 accumulator columns per thread fit the register file of 320 threads
  constexpr int kConv = BN == 128 ? 4 : 8;
  if (a.a_res) return launch_cfg<BN, kConv, true>(st, a.tmF, a.tmB, prm, grid, smem);
  return launch_cfg<BN, kConv, false>(st, a.tmF, a.tmB, prm, grid, smem);
}

}  // namespace

bool ozt_supported(int K, int bn, bool a_res, bool fold) {
  // K % 16: whole 16-wide MMA k steps (the float32 boxes past K read zeros); K > 32 when K is
  // not a multiple of 32: a warp's rows then reach at most two rows of the next stage
  if (K % 16 != 0 || (K % 32 != 0 && K < 48) || (bn != 32 && bn != 48 && bn != 64 && bn != 128) || K % bn != 0)
    return false;
  if (fold && (K % 128 != 0 || (K / 2) % bn != 0)) return false;
  const OztConfig c = ozt_config(bn, fold ? K / 2 : K, a_res);
  return c.nat >= 1 && c.nacc >= (bn == 128 ? 1 : 2) && c.a_col0 + c.nat * c.at_cols <= 512 && c.sb >= 2 &&
         c.smem <= 227 * 1024;
}

cudaError_t launch_mp_ozt(kpme_plan_t P, const OztArgs& a) {
  const int bn = P->tc_bn;
  const int kc = a.fold ? a.Kr / 2 : a.Kr;
  const OztConfig c = ozt_config(bn, kc, a.a_res);
  // one converter thread per row (four converter warps, BN = 128) and every chunk of a unit
  // staged at once: the converters take the rows' powers of two themselves
  const int kchunks_ = (kc + kChunk - 1) / kChunk;
  if (a.self_max && !(bn == 128 && kchunks_ <= c.sf)) return cudaErrorInvalidValue;
  OztParams prm{};
  prm.M = a.M;
  prm.N = a.N;
  prm.Kr = a.Kr;
  prm.kc = kc;
  prm.fold = a.fold ? 1 : 0;
  prm.self_max = a.self_max ? 1 : 0;
  prm.tile_max = a.tile_max ? 1 : 0;
  if (a.tile_max && !(bn == 128 && a.fold && a.Kr == 2 * kBM && (a.a_res ? a.rowmax_out : a.rowmax_in)))
    return cudaErrorInvalidValue;
  prm.kchunks = (kc + kChunk - 1) / kChunk;
  prm.sb = c.sb;
  prm.bstage = kSlices * bn * 128;
  prm.sf = c.sf;
  prm.nacc = c.nacc;
  prm.nat = c.nat;
  prm.a_col0 = c.a_col0;
  prm.at_cols = c.at_cols;
  prm.mode = a.mode;
  prm.rowmax_in = a.rowmax_in;
  prm.rm_in_bs = a.rm_in_bs;
  prm.out = a.out;
  prm.out_bs = a.out_bs;
  prm.out_base = a.out_base;
  prm.rowmax_out = a.rowmax_out;
  prm.rm_out_bs = a.rm_out_bs;
  prm.start = a.jobs->d_start;
  prm.pairs = a.jobs->d_pairs;
  prm.n_jobs = a.jobs->n_jobs;
  prm.status = P->d_status;
  prm.wait_cycles = P->wait_cycles;
  prm.n_pairs = (int)a.jobs->h_pairs.size();
  const int smem = c.smem + prm.n_pairs * (int)sizeof(int2) + (prm.n_jobs + 1) * (int)sizeof(int);
  if (smem > 227 * 1024) return cudaErrorInvalidValue;
  const int items = ((a.M + kBM - 1) / kBM) * (a.N / bn) * a.jobs->n_jobs;
  dim3 grid(items < P->sm_count ? items : P->sm_count);
  switch (bn) {
    case 32: return launch_bn<32>(a, P->stream, prm, grid, smem);
    case 128: return launch_bn<128>(a, P->stream, prm, grid, smem);
    case 48: return launch_bn<48>(a, P->stream, prm, grid, smem);
    case 64: return launch_bn<64>(a, P->stream, prm, grid, smem);
    default: return cudaErrorInvalidValue;
  }
}

// The reflection basis of a K^3 mesh (K even).  On each axis the mirror points a and K - 1 - a
// (a < K/2) are replaced by their sum (stored at a) and difference (stored at K - 1 - a); one
// thread takes the octet of mirror points of (a1, a2, a3), reads its eight values, applies the
// butterfly on the three axes in double-float arithmetic (float32 pairs: the float64 pipe of
// this GPU would bound the pass) and writes the eight results, rounded once to float32.  The
// unfolding applies the same butterfly and the factor 1/8 (the butterfly squared is twice the
// identity per axis); it reads and writes the same octet, so it runs in place.
__device__ __forceinline__ df df_of(float v) { return {v, 0.0f}; }
__device__ __forceinline__ df df_of(double v) { return df_from(v); }
__device__ __forceinline__ df df_neg(df a) { return {-a.hi, -a.lo}; }

template <typename TIN, bool UNFOLD>
__global__ void fold_mesh_kernel(const TIN* in, float* out, int K, float* __restrict__ zero, int64_t nz) {
  const int h = K / 2;
  const int64_t n_oct = (int64_t)h * h * h;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < n_oct; o += stride) {
    const int a3 = (int)(o % h), a2 = (int)((o / h) % h), a1 = (int)(o / ((int64_t)h * h));
    const int p1[2] = {a1, K - 1 - a1}, p2[2] = {a2, K - 1 - a2}, p3[2] = {a3, K - 1 - a3};
    df v[2][2][2];
#pragma unroll
    for (int s1 = 0; s1 < 2; ++s1)
#pragma unroll
      for (int s2 = 0; s2 < 2; ++s2)
#pragma unroll
        for (int s3 = 0; s3 < 2; ++s3) v[s1][s2][s3] = df_of(in[((int64_t)p1[s1] * K + p2[s2]) * K + p3[s3]]);
    // one axis after the other (each butterfly reads values the previous axis finished)
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const df a = v[i][j][0], b = v[i][j][1];
        v[i][j][0] = df_add(a, b);
        v[i][j][1] = df_add(a, df_neg(b));
      }
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const df a = v[i][0][j], b = v[i][1][j];
        v[i][0][j] = df_add(a, b);
        v[i][1][j] = df_add(a, df_neg(b));
      }
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const df a = v[0][i][j], b = v[1][i][j];
        v[0][i][j] = df_add(a, b);
        v[1][i][j] = df_add(a, df_neg(b));
      }
    const float scale = UNFOLD ? 0.125f : 1.0f;   // a power of two: exact
#pragma unroll
    for (int s1 = 0; s1 < 2; ++s1)
#pragma unroll
      for (int s2 = 0; s2 < 2; ++s2)
#pragma unroll
        for (int s3 = 0; s3 < 2; ++s3)
          out[((int64_t)p1[s1] * K + p2[s2]) * K + p3[s3]] =
              scale * __fadd_rn(v[s1][s2][s3].hi, v[s1][s2][s3].lo);
  }
  if (zero)
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nz; i += stride) zero[i] = 0.0f;
}

cudaError_t launch_fold_mesh(kpme_plan_t P, const void* in, bool in_double, float* out, int K, float* zero,
                             int64_t nz) {
  const int64_t n_oct = (int64_t)(K / 2) * (K / 2) * (K / 2);
  const int threads = 256;
  const int64_t want = (std::max<int64_t>(n_oct, nz) + threads - 1) / threads;
  const int grid = (int)std::min<int64_t>(std::max<int64_t>(want, 1), (int64_t)P->sm_count * 16);
  if (in_double)
    fold_mesh_kernel<double, false><<<grid, threads, 0, P->stream>>>((const double*)in, out, K, zero, nz);
  else
    fold_mesh_kernel<float, false><<<grid, threads, 0, P->stream>>>((const float*)in, out, K, zero, nz);
  return cudaGetLastError();
}

cudaError_t launch_unfold_mesh(kpme_plan_t P, float* mesh, int K) {
  const int64_t n_oct = (int64_t)(K / 2) * (K / 2) * (K / 2);
  const int threads = 256;
  const int grid = (int)std::min<int64_t>((n_oct + threads - 1) / threads, (int64_t)P->sm_count * 16);
  fold_mesh_kernel<float, true><<<grid, threads, 0, P->stream>>>(mesh, mesh, K, nullptr, 0);
  return cudaGetLastError();
}

cudaError_t launch_rowmax_rows(kpme_plan_t P, const float* in, int64_t rows, int K, float* out, float* zero,
                               int64_t nz) {
  if (rows <= 0) return zero && nz > 0 ? cudaMemsetAsync(zero, 0, (size_t)nz * sizeof(float), P->stream) : cudaSuccess;
  const int threads = 256;
  const int64_t blocks = (rows * 32 + threads - 1) / threads;
  rowmax_rows_kernel<<<(unsigned)blocks, threads, 0, P->stream>>>(in, rows, K, out, zero, nz);
  return cudaGetLastError();
}

}  // namespace kpme
