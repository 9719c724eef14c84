// k_finalize.cu -- integration end: baseline weights and normalisation.
//
// W_ab counts the FFT blocks of the integration that are valid at both
// stations a and b; blocks valid at only one end were stored as zero spectra
// and so add nothing to V_ab.  The output is V_ab / (W_ab * N) (zero when
// W_ab = 0), which puts the autocorrelation of 2-bit data at the mean power of
// the quantised levels.  The KZ partial accumulators are summed in a fixed
// order.
#include "corr_internal.cuh"

namespace corr {

__global__ void k_weights(FinParams p) {
  const int bl = blockIdx.x;
  // decode baseline index -> (a, b)
  int a = 0, q = bl;
  while (q >= p.S - a) { q -= p.S - a; ++a; }
  const int b = a + q;
  const uint8_t* va = p.valid + (size_t)a * p.ld;
  const uint8_t* vb = p.valid + (size_t)b * p.ld;
  int cnt = 0;
  for (int i = threadIdx.x; i < p.M; i += blockDim.x) cnt += (va[i] && vb[i]) ? 1 : 0;
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, o);
  __shared__ int ws[32];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = cnt;
  __syncthreads();
  if (threadIdx.x == 0) {
    int tot = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += ws[w];
    p.wcount[bl] = tot;
    if (p.weights) p.weights[bl] = (double)tot;
  }
}

cudaError_t launch_weights(const FinParams& p, cudaStream_t s) {
  k_weights<<<nbl_of(p.S), 256, 0, s>>>(p);
  return cudaGetLastError();
}

__global__ void k_finalize(FinParams p) {
  const size_t per = (size_t)p.G * p.nchan;
  const size_t total = (size_t)nbl_of(p.S) * per;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  const bool failed = p.err && *p.err != 0;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += stride) {
    const int bl = (int)(e / per);
    float2 v = make_float2(0.f, 0.f);
    for (int kz = 0; kz < p.KZ; ++kz) {
      const float2 x = p.part[(size_t)kz * total + e];
      v.x += x.x;
      v.y += x.y;
    }
    const int w = p.wcount[bl];
    const float sc = w > 0 ? (float)((double)p.unscale / ((double)w * (double)p.N)) : 0.f;
    p.out[e] = failed ? make_float2(__int_as_float(0x7fc00000), __int_as_float(0x7fc00000))
                      : make_float2(v.x * sc, v.y * sc);
  }
}

cudaError_t launch_finalize(const FinParams& p, cudaStream_t s) {
  const size_t total = (size_t)nbl_of(p.S) * p.G * p.nchan;
  int blocks = (int)((total + 255) / 256);
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (blocks < 1) blocks = 1;
  k_finalize<<<blocks, 256, 0, s>>>(p);
  return cudaGetLastError();
}

// Tensor-core partial sums are laid out [KZ][G][nchan][nbl] (baseline
// fastest, as the X kernel's epilogue writes them).
__global__ void k_finalize_tc(FinParams p, float unscale) {
  const int nbl = nbl_of(p.S);
  const size_t per = (size_t)p.G * p.nchan;
  const size_t total = (size_t)nbl * per;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += stride) {
    const int bl = (int)(e / per);
    const size_t gk = e - (size_t)bl * per;  // g * nchan + k
    float2 v = make_float2(0.f, 0.f);
    for (int kz = 0; kz < p.KZ; ++kz) {
      const float2 x = p.part[((size_t)kz * per + gk) * nbl + bl];
      v.x += x.x;
      v.y += x.y;
    }
    const int w = p.wcount[bl];
    const float sc = w > 0 ? (float)((double)unscale / ((double)w * (double)p.N)) : 0.f;
    p.out[e] = make_float2(v.x * sc, v.y * sc);
  }
}

cudaError_t launch_finalize_tc(const FinParams& p, float unscale, cudaStream_t s) {
  const size_t total = (size_t)nbl_of(p.S) * p.G * p.nchan;
  int blocks = (int)((total + 255) / 256);
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (blocks < 1) blocks = 1;
  k_finalize_tc<<<blocks, 256, 0, s>>>(p, unscale);
  return cudaGetLastError();
}

// Both hands of two polarisations.  The X step ran over 2S virtual stations
// v = pol * S + station per subband, so V_ab^pq is the virtual product
// P[p S + a][q S + b] when p S + a <= q S + b and its conjugate otherwise
// (for a = b and pq = 10: the conjugate of the 01 product).
template <bool TC>
__global__ void k_finalize_cross(FinParams p, float unscale) {
  const int S = p.S, S2 = 2 * S, nsub = p.G, nch = p.nchan;
  const int nblv = nbl_of(S2);
  const size_t total = (size_t)nbl_of(S) * nsub * 4 * nch;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += stride) {
    const int k = (int)(e % nch);
    size_t r = e / nch;
    const int pq = (int)(r & 3);
    r >>= 2;
    const int sb = (int)(r % nsub);
    const int bl = (int)(r / nsub);
    int a = 0, q = bl;
    while (q >= S - a) { q -= S - a; ++a; }
    const int b = a + q;
    int v1 = (pq >> 1) * S + a, v2 = (pq & 1) * S + b;
    const bool flip = v1 > v2;
    if (flip) {
      const int t = v1;
      v1 = v2;
      v2 = t;
    }
    const int blv = bl_index(v1, v2, S2);
    float2 v = make_float2(0.f, 0.f);
    for (int kz = 0; kz < p.KZ; ++kz) {
      const float2 x = TC ? p.part[(((size_t)kz * nsub + sb) * nch + k) * nblv + blv]
                          : p.part[(((size_t)kz * nblv + blv) * nsub + sb) * nch + k];
      v.x += x.x;
      v.y += x.y;
    }
    if (flip) v.y = -v.y;
    const int w = p.wcount[bl];
    const float sc = w > 0 ? (float)((double)unscale / ((double)w * (double)p.N)) : 0.f;
    p.out[e] = make_float2(v.x * sc, v.y * sc);
  }
}

cudaError_t launch_finalize_cross(const FinParams& p, bool tc, float unscale, cudaStream_t s) {
  const size_t total = (size_t)nbl_of(p.S) * p.G * 4 * p.nchan;
  int blocks = (int)((total + 255) / 256);
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (blocks < 1) blocks = 1;
  if (tc)
    k_finalize_cross<true><<<blocks, 256, 0, s>>>(p, unscale);
  else
    k_finalize_cross<false><<<blocks, 256, 0, s>>>(p, unscale);
  return cudaGetLastError();
}

}  // namespace corr
