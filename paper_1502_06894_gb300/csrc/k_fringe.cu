// k_fringe.cu -- delay-rate fringe search of one baseline's visibilities
// (the wide-window fringe search the paper lists for RadioAstron, Sec. 2).
//
// For visibilities V[t][k] (t: sub-integration, k: channel) the map is the
// zero-padded two-dimensional inverse DFT, unnormalised,
//     M[r][l] = sum_t sum_k V[t][k] exp(+2 pi i (k l / Nd + t r / Nr)),
// and the peak is the largest |M|, the smaller flat index r * Nd + l on ties.
// Two passes of a shared-memory radix-2 complex FFT (one CTA per transform):
// over channels for every sub-integration (written transposed, lag-major),
// then over sub-integrations for every lag; then one reduction for the peak.
#include "../../include/corr.h"
#include "corr_internal.cuh"

#include <math.h>
#include <stdint.h>
#include <string.h>

namespace corr {

namespace {

constexpr int kFftThreads = 512;
constexpr int kMaxFft = 16384;

__device__ __forceinline__ int bitrev(int x, int bits) { return (int)(__brev((unsigned)x) >> (32 - bits)); }

// One inverse transform of length n (a power of two) per CTA: row `row` of
// `in` (in_len values, the rest zero) -> out[row * orow + i * ocol], i < n.
// Iterative radix-2 decimation in time on a bit-reversed copy in shared
// memory; the twiddles exp(+2 pi i j / n), j < n/2, come from sincospif.
__global__ void __launch_bounds__(kFftThreads) k_cfft_inv(const float2* __restrict__ in, int in_len, int64_t in_ld,
                                                          float2* __restrict__ out, int n, int logn, int64_t orow,
                                                          int64_t ocol) {
  extern __shared__ __align__(16) float2 sm[];
  float2* s = sm;          // [n]
  float2* tw = sm + n;     // [n / 2]
  const int row = blockIdx.x;
  const float2* src = in + (int64_t)row * in_ld;
  for (int j = threadIdx.x; j < n / 2; j += blockDim.x) {
    float sn, cs;
    sincospif(2.0f * (float)j / (float)n, &sn, &cs);
    tw[j] = make_float2(cs, sn);
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const int j = bitrev(i, logn);
    s[i] = j < in_len ? src[j] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  for (int half = 1; half < n; half <<= 1) {
    const int step = n / (2 * half);  // twiddle index stride for this stage
    for (int b = threadIdx.x; b < n / 2; b += blockDim.x) {
      const int p = b & (half - 1);
      const int i0 = ((b - p) << 1) + p;
      const int i1 = i0 + half;
      const float2 w = tw[p * step];
      const float2 u = s[i0], x = s[i1];
      const float2 v = make_float2(x.x * w.x - x.y * w.y, x.x * w.y + x.y * w.x);
      s[i0] = make_float2(u.x + v.x, u.y + v.y);
      s[i1] = make_float2(u.x - v.x, u.y - v.y);
    }
    __syncthreads();
  }
  float2* dst = out + (int64_t)row * orow;
  for (int i = threadIdx.x; i < n; i += blockDim.x) dst[(int64_t)i * ocol] = s[i];
}

// Largest amplitude with the smallest flat index on ties: one 64-bit key per
// element, amplitude bits (non-negative floats order like their bit
// patterns) above the complement of the index, reduced with atomicMax.
__global__ void __launch_bounds__(256) k_fringe_peak(const float2* __restrict__ map, int64_t count,
                                                     unsigned long long* __restrict__ best) {
  unsigned long long key = 0ull;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x) {
    const float2 v = map[e];
    const float a = sqrtf(v.x * v.x + v.y * v.y);
    const unsigned long long k =
        ((unsigned long long)__float_as_uint(a) << 32) | (unsigned long long)(0xFFFFFFFFu - (uint32_t)e);
    key = k > key ? k : key;
  }
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long other = __shfl_down_sync(0xffffffffu, key, o);
    key = other > key ? other : key;
  }
  __shared__ unsigned long long ws[8];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = key;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) key = ws[w] > key ? ws[w] : key;
    atomicMax(best, key);
  }
}

int ilog2_exact(int n) {
  if (n < 2 || (n & (n - 1))) return -1;
  int l = 0;
  while ((1 << l) < n) ++l;
  return l;
}

}  // namespace

}  // namespace corr

using namespace corr;

extern "C" int corr_fringe_search(const float* dev_vis, int nsub, int nchan, int pad_rate, int pad_delay,
                                  float* dev_map, int* peak_rate, int* peak_lag, float* peak_amp,
                                  float* peak_value, void* cuda_stream) {
  if (!dev_vis || !dev_map || nsub < 1 || nchan < 1) return CORR_EINVAL;
  const int lr = ilog2_exact(pad_rate), ld = ilog2_exact(pad_delay);
  if (lr < 0 || ld < 0 || pad_rate < nsub || pad_delay < nchan || pad_rate > kMaxFft || pad_delay > kMaxFft ||
      (int64_t)pad_rate * pad_delay > ((int64_t)1 << 26))
    return CORR_EINVAL;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const float2* V = reinterpret_cast<const float2*>(dev_vis);
  float2* M = reinterpret_cast<float2*>(dev_map);
  // scratch: the lag transforms, lag-major [pad_delay][nsub], plus the peak key
  const size_t scratch = sizeof(float2) * (size_t)pad_delay * nsub + 256;
  void* buf = nullptr;
  if (cudaMallocAsync(&buf, scratch, st) != cudaSuccess) {
    cudaGetLastError();
    return CORR_ENOMEM;
  }
  float2* X1 = reinterpret_cast<float2*>(buf);
  unsigned long long* best =
      reinterpret_cast<unsigned long long*>(reinterpret_cast<char*>(buf) + sizeof(float2) * (size_t)pad_delay * nsub);
  cudaError_t e = cudaSuccess;
  const int maxn = pad_rate > pad_delay ? pad_rate : pad_delay;
  const size_t smem_max = sizeof(float2) * ((size_t)maxn + maxn / 2);
  e = cudaFuncSetAttribute(k_cfft_inv, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max);
  // over channels: row t of V -> X1[l][t]
  if (e == cudaSuccess) {
    const int thr = pad_delay / 2 < kFftThreads ? (pad_delay / 2 > 32 ? pad_delay / 2 : 32) : kFftThreads;
    k_cfft_inv<<<nsub, thr, sizeof(float2) * ((size_t)pad_delay + pad_delay / 2), st>>>(V, nchan, nchan, X1,
                                                                                        pad_delay, ld, 1, nsub);
    e = cudaGetLastError();
  }
  // over sub-integrations: row l of X1 -> M[r][l]
  if (e == cudaSuccess) {
    const int thr = pad_rate / 2 < kFftThreads ? (pad_rate / 2 > 32 ? pad_rate / 2 : 32) : kFftThreads;
    k_cfft_inv<<<pad_delay, thr, sizeof(float2) * ((size_t)pad_rate + pad_rate / 2), st>>>(X1, nsub, nsub, M,
                                                                                          pad_rate, lr, 1, pad_delay);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(best, 0, sizeof(unsigned long long), st);
  const int64_t count = (int64_t)pad_rate * pad_delay;
  if (e == cudaSuccess) {
    int blocks = (int)((count + 255) / 256);
    if (blocks > 152 * 8) blocks = 152 * 8;
    k_fringe_peak<<<blocks, 256, 0, st>>>(M, count, best);
    e = cudaGetLastError();
  }
  unsigned long long key = 0ull;
  float2 pv = make_float2(0.f, 0.f);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&key, best, sizeof(key), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  const int64_t idx = (int64_t)(0xFFFFFFFFu - (uint32_t)(key & 0xFFFFFFFFull));
  if (e == cudaSuccess && (idx < 0 || idx >= count)) e = cudaErrorUnknown;
  if (e == cudaSuccess) e = cudaMemcpy(&pv, M + idx, sizeof(float2), cudaMemcpyDeviceToHost);
  cudaFreeAsync(buf, st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return CORR_ECUDA;
  }
  if (peak_rate) *peak_rate = (int)(idx / pad_delay);
  if (peak_lag) *peak_lag = (int)(idx % pad_delay);
  if (peak_amp) {
    const uint32_t bits = (uint32_t)(key >> 32);
    memcpy(peak_amp, &bits, sizeof(float));
  }
  if (peak_value) {
    peak_value[0] = pv.x;
    peak_value[1] = pv.y;
  }
  return CORR_OK;
}
