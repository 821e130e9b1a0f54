// CUDA-core mode products (the float64 and float32 forms of the SKP contraction).
//
// One launch computes, for every job j,
//     out[j][n][m] (+)= sum_{(a, f) in pairs(j)} sum_k fac[f][n][k] * in[a][m][k]
// i.e. the reshaped Kronecker step of Algorithm 2 (§3.3): the input tensor is viewed as
// an M x Kr matrix whose rows are all indices but the contracted one (contiguous), the
// factor as N x Kr, and the product is stored transposed so that the new index becomes
// the slowest.  Three such steps rotate [k1][k2][k3] -> [k3'][k1][k2] -> [k2'][k3'][k1]
// -> [k1'][k2'][k3'], so no explicit permutation (Algorithm 1's Q^left / Q^right) is needed.
#include "kpme_internal.cuh"

namespace kpme {
namespace {

constexpr int BK = 16;

// BM x BN tile per CTA of THREADS threads, each computing TM x TN outputs:
// (64, 64, 256 threads, 4 x 4) for large grids, (32, 32, 64 threads, 4 x 4) for small ones.
template <typename T, int BM, int BN, int THREADS>
__global__ void __launch_bounds__(THREADS) mp_simt_kernel(const T* __restrict__ in, int64_t in_bs,
                                                          const T* __restrict__ fac, T* __restrict__ out,
                                                          int64_t out_bs, int M, int N, int Kr,
                                                          const int* __restrict__ start,
                                                          const int2* __restrict__ pairs, int mode) {
  constexpr int TM = 4, TN = 4, TX = BM / TM;
  __shared__ T As[BK][BM + 1];
  __shared__ T Bs[BK][BN + 1];
  const int job = blockIdx.z;
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
  const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
  T acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = T(0);

  const int p0 = start[job], p1 = start[job + 1];
  for (int p = p0; p < p1; ++p) {
    const int2 pr = pairs[p];
    const T* A = in + (int64_t)pr.x * in_bs;
    const T* B = fac + (int64_t)pr.y * N * Kr;
    for (int k0 = 0; k0 < Kr; k0 += BK) {
      // 64 x 16 tiles, 4 elements per thread, k fastest (coalesced rows)
#pragma unroll
      for (int r = 0; r < (BM * BK) / THREADS; ++r) {
        const int idx = threadIdx.x + r * THREADS;
        const int row = idx / BK, kk = idx % BK;
        const int gm = m0 + row, gk = k0 + kk;
        As[kk][row] = (gm < M && gk < Kr) ? A[(int64_t)gm * Kr + gk] : T(0);
        const int gn = n0 + row;
        Bs[kk][row] = (gn < N && gk < Kr) ? B[(int64_t)gn * Kr + gk] : T(0);
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < BK; ++kk) {
        T a[TM], b[TN];
#pragma unroll
        for (int i = 0; i < TM; ++i) a[i] = As[kk][tx + TX * i];
#pragma unroll
        for (int j = 0; j < TN; ++j) b[j] = Bs[kk][ty + (BN / TN) * j];
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
          for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
      }
      __syncthreads();
    }
  }
  T* O = out + (mode == 0 ? (int64_t)job * out_bs : 0);
#pragma unroll
  for (int j = 0; j < TN; ++j) {
    const int n = n0 + ty + (BN / TN) * j;
    if (n >= N) continue;
#pragma unroll
    for (int i = 0; i < TM; ++i) {
      const int m = m0 + tx + TX * i;
      if (m >= M) continue;
      T* dst = O + (int64_t)n * M + m;
      if (mode == 0)
        *dst = acc[i][j];
      else
        atomicAdd(dst, acc[i][j]);
    }
  }
}

}  // namespace

template <int BM, int BN, int THREADS>
cudaError_t launch_tiles(bool dbl, const void* in, int64_t in_bs, const void* fac, void* out, int64_t out_bs, int M,
                         int N, int Kr, const JobList& jobs, int mode, cudaStream_t s) {
  dim3 grid((M + BM - 1) / BM, (N + BN - 1) / BN, jobs.n_jobs);
  if (dbl)
    mp_simt_kernel<double, BM, BN, THREADS><<<grid, THREADS, 0, s>>>(
        (const double*)in, in_bs, (const double*)fac, (double*)out, out_bs, M, N, Kr, jobs.d_start, jobs.d_pairs, mode);
  else
    mp_simt_kernel<float, BM, BN, THREADS><<<grid, THREADS, 0, s>>>(
        (const float*)in, in_bs, (const float*)fac, (float*)out, out_bs, M, N, Kr, jobs.d_start, jobs.d_pairs, mode);
  return cudaGetLastError();
}

cudaError_t launch_mp_simt(bool dbl, const void* in, int64_t in_bs, const void* fac, void* out, int64_t out_bs,
                           int M, int N, int Kr, const JobList& jobs, int mode, cudaStream_t s) {
  const int64_t big = (int64_t)((M + 63) / 64) * ((N + 63) / 64) * jobs.n_jobs;
  if (big >= 4 * 152) return launch_tiles<64, 64, 256>(dbl, in, in_bs, fac, out, out_bs, M, N, Kr, jobs, mode, s);
  return launch_tiles<32, 32, 64>(dbl, in, in_bs, fac, out, out_bs, M, N, Kr, jobs, mode, s);
}

}  // namespace kpme
