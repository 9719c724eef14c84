// corr_static.cu -- corr_correlate_static: one integration of the FX path
// without any device allocation, for callers that cannot call cudaMalloc.
//
// The handle API (corr_create ... corr_correlate_device) allocates its work
// buffers on the device.  Some callers cannot allow that: a host program that
// owns a fixed device-memory budget and forbids libraries to allocate after
// start-up, or a real-time pipeline that must not call cudaMalloc/cudaFree on
// its hot path because those calls can synchronise the whole device and stall
// its other streams.  This entry point runs the same kernels (delay blocks,
// F, X, weights, finalise) with every intermediate -- the delay model, the
// block descriptors, the spectra of one chunk and the X partial sums -- placed
// in one file-scope device array of fixed size, kStaticScratchBytes.  Every
// GPU that loads the library holds that array until the process exits.
#include "../../include/corr.h"
#include "corr_internal.cuh"

#include <math.h>

#include <mutex>

using namespace corr;

namespace {

constexpr size_t kStaticScratchBytes = (size_t)64 << 20;  // 64 MiB, documented in corr.h
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

// Device address of g_static_scratch per device, and the context it was
// resolved in (a cudaDeviceReset gives the device a new context, whose copy
// of the array may sit elsewhere).
unsigned char* g_scratch_ptr[kMaxDevices];
unsigned long long g_scratch_ctx[kMaxDevices];
std::mutex g_static_mu;

// Errors are reported by return code only (no handle to hold a message).
int set_err(int code, const char*) { return code; }

// Once per device (and context), with that device current: resolve the
// array's device address (its host-side name is only a stand-in) and load the
// FFT constants.
int static_setup(int dev, unsigned char** out) {
  std::lock_guard<std::mutex> lk(g_static_mu);
  const unsigned long long ctx = current_context_id();
  if (!g_scratch_ptr[dev] || ctx == 0 || ctx != g_scratch_ctx[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return set_err(CORR_ECUDA, "corr_correlate_static: cudaGetSymbolAddress of the scratch array failed");
    }
    e = fstage_ensure_constants();
    if (e != cudaSuccess) {
      cudaGetLastError();
      return set_err(CORR_ECUDA, "corr_correlate_static: loading FFT constants failed");
    }
    g_scratch_ptr[dev] = (unsigned char*)p;
    g_scratch_ctx[dev] = current_context_id();
  }
  *out = g_scratch_ptr[dev];
  return CORR_OK;
}

// Small inputs that the call derives on the host go to the scratch as kernel
// parameters (copied at launch), not as copies from host memory that the
// call frees when it returns: up to kViewsPerLaunch station views per launch,
// and the FFT twiddles W_N^m = exp(-2 pi i m / N), computed in FP64 on the
// device and rounded to FP32.
constexpr int kViewsPerLaunch = 48;
struct ViewBatch {
  StationView v[kViewsPerLaunch];
};

__global__ void k_static_views(ViewBatch b, int n, StationView* dst) {
  const int i = threadIdx.x;
  if (i < n) dst[i] = b.v[i];
}

__global__ void k_static_twiddles(float2* tw, int N) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= N) return;
  double sn, cs;
  sincospi(-2.0 * (double)m / (double)N, &sn, &cs);
  tw[m] = make_float2((float)cs, (float)sn);
}

struct Carve {
  size_t off = 0;
  size_t take(size_t bytes) {
    size_t o = off;
    off += (bytes + 255) & ~(size_t)255;
    return o;
  }
};

}  // namespace

extern "C" int corr_correlate_static(const corr_scan_desc* d, int64_t integration, float* dev_out,
                                     double* dev_weights, void* cuda_stream) {
  if (!d || !dev_out) return set_err(CORR_EINVAL, "corr_correlate_static: desc and dev_out are required");
  const int S = d->stations, nsub = d->subbands, npol = d->pols, nchan = d->nchan;
  if (S < 1 || S > kMaxStations || npol < 1 || npol > 2 || nsub < 1 || nsub * npol > 32 ||
      !fstage_supported(nchan) || integration < 0)
    return set_err(CORR_EINVAL, "corr_correlate_static: bad shape (stations, subbands*pols <= 32, nchan)");
  if (!d->nu0_hz || !d->nseg || !d->seg_t0 || !d->seg_coeffs || !d->dev_bytes || !d->nbytes || !d->first_sample)
    return set_err(CORR_EINVAL, "corr_correlate_static: a descriptor array is NULL");
  const int G = nsub * npol, N = 2 * nchan, nbl = nbl_of(S);
  const double spi_d = d->fs_hz * d->tint_s;
  const int64_t spi = llround(spi_d);
  if (!(d->fs_hz > 0) || fabs(spi_d - (double)spi) > 1e-6 || spi < N)
    return set_err(CORR_EINVAL, "corr_correlate_static: fs*tint must be a whole number of samples >= 2*nchan");
  for (int s = 0; s < S; ++s) {
    if (d->nseg[s] < 1 || d->nseg[s] > kMaxSegs)
      return set_err(CORR_EINVAL, "corr_correlate_static: each station needs 1..64 delay segments");
    if (!d->dev_bytes[s] || ((uintptr_t)d->dev_bytes[s] & 15) || (d->nbytes[s] & 3))
      return set_err(CORR_EINVAL, "corr_correlate_static: station bytes must be 16-byte aligned, a multiple of 4");
  }
  const int64_t bfirst = (integration * spi + N - 1) / N;
  const int M = (int)((((integration + 1) * spi + N - 1) / N) - bfirst);

  // ---- scratch layout; pick the largest chunk that fits ----
  Carve c;
  const size_t o_views = c.take(sizeof(StationView) * S);
  const size_t o_nseg = c.take(sizeof(int) * S);
  const size_t o_t0 = c.take(sizeof(double) * S * kMaxSegs);
  const size_t o_c = c.take(sizeof(double) * S * kMaxSegs * 6);
  const size_t o_nu0 = c.take(sizeof(double) * nsub);
  const size_t o_tw = c.take(sizeof(float2) * N);
  const size_t o_start = c.take(sizeof(int64_t) * (size_t)S * M);
  const size_t o_delta = c.take(sizeof(float) * (size_t)S * M);
  const size_t o_phi = c.take(sizeof(float) * (size_t)S * nsub * M);
  const size_t o_valid = c.take((size_t)S * M);
  const size_t o_wc = c.take(sizeof(int) * nbl);
  const size_t o_err = c.take(sizeof(int));
  const size_t fixed = c.off;
  const size_t per_block = sizeof(float2) * (size_t)G * S * nchan;
  const size_t per_part = sizeof(float2) * (size_t)nbl * G * nchan;
  int CB = M, KZ = 0;
  for (; CB >= 1; CB = (CB > 1) ? CB / 2 : 0) {
    KZ = xstage_kz(CB, S, G, nchan);
    const size_t need = fixed + ((per_block * CB + 255) & ~(size_t)255) + ((per_part * KZ + 255) & ~(size_t)255);
    if (need <= kStaticScratchBytes) break;
  }
  if (CB < 1)
    return set_err(CORR_ETOOBIG, "corr_correlate_static: this shape needs more than the 64 MiB static scratch");
  const size_t o_spec = c.take(per_block * CB);
  const size_t o_part = c.take(per_part * KZ);

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return set_err(CORR_ECUDA, "corr_correlate_static: no current CUDA device");
  }
  unsigned char* base = nullptr;
  int rc = static_setup(dev, &base);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)cuda_stream;

  // ---- small inputs into the scratch: the caller's descriptor arrays by
  //      copies from host memory, the rest by kernels with by-value parameters ----
  cudaError_t e = cudaSuccess;
  for (int s0 = 0; s0 < S && e == cudaSuccess; s0 += kViewsPerLaunch) {
    ViewBatch vb;
    const int n = (S - s0 < kViewsPerLaunch) ? S - s0 : kViewsPerLaunch;
    for (int q = 0; q < n; ++q) {
      const int s = s0 + q;
      vb.v[q].words = (const uint32_t*)d->dev_bytes[s];
      vb.v[q].nwords = (int64_t)(d->nbytes[s] / 4);
      vb.v[q].sample0 = d->first_sample[s];
      vb.v[q].ngroups = (int64_t)((d->nbytes[s] * 4) / (size_t)G);
      vb.v[q].host = 0;
      vb.v[q].payload = 0;
      vb.v[q].frame_ok = nullptr;
      vb.v[q].nframes = 0;
    }
    k_static_views<<<1, kViewsPerLaunch, 0, st>>>(vb, n, (StationView*)(base + o_views) + s0);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    k_static_twiddles<<<(N + 255) / 256, 256, 0, st>>>((float2*)(base + o_tw), N);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(base + o_nseg, d->nseg, sizeof(int) * S, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(base + o_t0, d->seg_t0, sizeof(double) * S * kMaxSegs, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(base + o_c, d->seg_coeffs, sizeof(double) * S * kMaxSegs * 6, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(base + o_nu0, d->nu0_hz, sizeof(double) * nsub, cudaMemcpyHostToDevice, st);
  // the X partial sums accumulate and the timeout flag latches, so both start
  // at zero on every call
  if (e == cudaSuccess) e = cudaMemsetAsync(base + o_part, 0, per_part * KZ, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(base + o_err, 0, sizeof(int), st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return set_err(CORR_ECUDA, "corr_correlate_static: writing inputs into the scratch failed");
  }

  // ---- the same kernels as the handle path ----
  DelayParams dp;
  dp.S = S;
  dp.nsub = nsub;
  dp.N = N;
  dp.G = G;
  dp.fs = d->fs_hz;
  dp.nseg = (const int*)(base + o_nseg);
  dp.seg_t0 = (const double*)(base + o_t0);
  dp.seg_c = (const double*)(base + o_c);
  dp.nu0 = (const double*)(base + o_nu0);
  dp.st = (const StationView*)(base + o_views);
  dp.b0 = bfirst;
  dp.nb = M;
  dp.ld = M;
  dp.start = (int64_t*)(base + o_start);
  dp.delta = (float*)(base + o_delta);
  dp.phi = (float*)(base + o_phi);
  dp.valid = (uint8_t*)(base + o_valid);
  dp.eps_out = nullptr;
  dp.tau_out = nullptr;
  dp.max_end = nullptr;
  dp.dphi = nullptr;
  e = launch_delay_blocks(dp, st);
  for (int c0 = 0; e == cudaSuccess && c0 < M; c0 += CB) {
    const int cb = (M - c0 < CB) ? (M - c0) : CB;
    FParams fp;
    fp.st = dp.st;
    fp.start = dp.start;
    fp.delta = dp.delta;
    fp.phi = dp.phi;
    fp.valid = dp.valid;
    fp.dphi = nullptr;
    fp.pre = 0;
    fp.cross = 0;
    fp.ld = M;
    fp.blk0 = c0;
    fp.CB = cb;
    fp.S = S;
    fp.G = G;
    fp.npol = npol;
    fp.nsub = nsub;
    fp.nchan = nchan;
    fp.lut0 = d->lut[0];
    fp.lut1 = d->lut[1];
    fp.lut2 = d->lut[2];
    fp.lut3 = d->lut[3];
    fp.twN = (const float2*)(base + o_tw);
    fp.out_kind = 0;
    fp.scale = 1.0f;
    fp.out = base + o_spec;
    e = launch_fstage(fp, st);
    if (e != cudaSuccess) break;
    XParams xp;
    xp.spec = (const float2*)(base + o_spec);
    xp.CB = cb;
    xp.S = S;
    xp.G = G;
    xp.nchan = nchan;
    xp.KZ = KZ;
    xp.part = (float2*)(base + o_part);
    xp.err = (int*)(base + o_err);
    e = launch_xstage(xp, st);
  }
  if (e == cudaSuccess) {
    FinParams fin;
    fin.part = (const float2*)(base + o_part);
    fin.KZ = KZ;
    fin.S = S;
    fin.G = G;
    fin.nchan = nchan;
    fin.N = N;
    fin.valid = dp.valid;
    fin.ld = M;
    fin.M = M;
    fin.wcount = (int*)(base + o_wc);
    fin.out = (float2*)dev_out;
    fin.weights = dev_weights;
    fin.err = (const int*)(base + o_err);  // a timed-out X-step wait turns the output into NaN
    e = launch_weights(fin, st);
    if (e == cudaSuccess) e = launch_finalize(fin, st);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    return set_err(CORR_ECUDA, cudaGetErrorString(e));
  }
  return CORR_OK;
}
