// k_delay.cu -- delay-block kernel: per (station, FFT block) the FP64 delay
// model, the integer-sample window start, the fractional-delay phase slope
// and the absolute fringe phase; plus a debug kernel that unpacks codes.
//
// The paper (Sec. 2) has the delay model server (Calc, extended to a moving,
// relativistic spacecraft and the spacecraft -> tracking-station leg) supply
// every station's delay.  It enters here as polynomial segments
// tau(t) = sum_i c_i (t - t0)^i in seconds, t relative to the scan epoch.
// FP64 is needed: a spacecraft delay near 1.2 s at 32 Msample/s is ~4e7
// samples, beyond the FP32 mantissa.
//
// Readings (the paper gives none of this):
//   block b spans geocentric samples [b*N, b*N + N), centre t_c = (b*N + N/2)/fs;
//   segment = largest t0 <= t_c; tau by Horner from c5 with fma at each step;
//   n_b = floor(fma(tau, fs, 0.5)); eps = tau - n_b/fs; the window starts at
//   station sample b*N + n_b; phi = frac(nu0 * tau) in turns.
// Every FP64 operation below is written with an explicit rounding intrinsic
// so that no multiply-add is contracted: the integer delay must come out
// bit-identical to a plain IEEE evaluation of the same sequence.
#include "corr_internal.cuh"

namespace corr {

__global__ void k_delay_blocks(DelayParams p) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int s = blockIdx.y;
  if (i >= p.nb) return;
  const int64_t b = p.b0 + i;
  const int N = p.N;
  const double tc = __ddiv_rn((double)(b * (int64_t)N + N / 2), p.fs);
  const double* t0 = p.seg_t0 + (size_t)s * kMaxSegs;
  const int ns = p.nseg[s];
  int seg = -1;
  for (int q = 0; q < ns; ++q)
    if (t0[q] <= tc) seg = q;
  const bool covered = seg >= 0;
  if (seg < 0) seg = 0;
  const double* c = p.seg_c + ((size_t)s * kMaxSegs + seg) * 6;
  const double u = __dsub_rn(tc, t0[seg]);
  double tau = c[5];
#pragma unroll
  for (int q = 4; q >= 0; --q) tau = __fma_rn(tau, u, c[q]);
  const int64_t n = (int64_t)floor(__fma_rn(tau, p.fs, 0.5));
  const double eps = __dsub_rn(tau, __ddiv_rn((double)n, p.fs));
  const int64_t start = b * (int64_t)N + n;
  const StationView v = p.st[s];
  const int64_t rel = start - v.sample0;
  bool ok = covered && rel >= 0 && rel + N <= v.ngroups;
  if (ok && v.payload > 0) {
    // framed input: every frame holding a byte of the window must be valid
    const int G = p.G;
    const int64_t qa = (2 * rel * G) >> 3, qb = (2 * (rel + N) * G - 1) >> 3;
    for (int64_t f = qa / v.payload; f <= qb / v.payload && ok; ++f) ok = f < v.nframes && v.frame_ok[f] != 0;
  }
  const size_t o = (size_t)s * p.ld + i;
  p.start[o] = start;
  p.valid[o] = ok ? 1 : 0;
  p.delta[o] = (float)__ddiv_rn(__dmul_rn(eps, p.fs), (double)N);
  // pre-F rotation: the delay rate at t_c (derivative of the same segment)
  double rate = 0.0;
  if (p.dphi) {
#pragma unroll
    for (int q = 5; q >= 1; --q) rate = __fma_rn(rate, u, (double)q * c[q]);
  }
  for (int sb = 0; sb < p.nsub; ++sb) {
    double ph = __dmul_rn(p.nu0[sb], tau);
    ph = __dsub_rn(ph, floor(ph));
    const size_t os = ((size_t)s * p.nsub + sb) * p.ld + i;
    if (p.dphi) {
      // phase step per sample (turns) and the phase at the block's first
      // sample, N/2 samples before the centre; the step splits into a part of
      // at most 10 significant bits (exact times any sample index < 2^14 in
      // FP32) and the rest
      const double step = p.nu0[sb] * rate / p.fs;
      double p0 = ph - step * (double)(N / 2);
      p0 -= floor(p0);
      double hi = 0.0;
      if (step != 0.0) {
        int ex = 0;
        frexp(step, &ex);
        hi = ldexp(rint(ldexp(step, 10 - ex)), ex - 10);
      }
      p.phi[os] = (float)p0;
      p.dphi[os] = make_float2((float)hi, (float)(step - hi));
    } else {
      p.phi[os] = (float)ph;
    }
  }
  if (p.eps_out) p.eps_out[o] = eps;
  if (p.tau_out) p.tau_out[o] = tau;
  if (p.max_end) {
    // [0]: max window end, [1]: min window start (both relative to the
    // station's first sample, offset by 2^62 so they order as unsigned);
    // [2]: number of valid blocks.
    const unsigned long long off = 1ull << 62;
    atomicMax(&p.max_end[3 * s + 0], (unsigned long long)(rel + N) + off);
    atomicMin(&p.max_end[3 * s + 1], (unsigned long long)rel + off);
    if (ok) atomicAdd(&p.max_end[3 * s + 2], 1ull);
  }
}

// Deframe: one CTA row per frame; the payload moves in 16-byte pieces (the
// payload and the frame length are multiples of 16 bytes).
__global__ void k_deframe(const uint8_t* __restrict__ raw, int payload, int64_t f0, int64_t f1,
                          uint8_t* __restrict__ out, uint8_t* __restrict__ frame_ok) {
  const int64_t f = f0 + blockIdx.y + (int64_t)gridDim.y * blockIdx.z;
  if (f >= f1) return;
  const uint8_t* fr = raw + f * (int64_t)(kFrameHeader + payload);
  const uint4* src = reinterpret_cast<const uint4*>(fr + kFrameHeader);
  uint4* dst = reinterpret_cast<uint4*>(out + f * (int64_t)payload);
  const int n16 = payload / 16;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n16; i += gridDim.x * blockDim.x) dst[i] = src[i];
  if (blockIdx.x == 0 && threadIdx.x == 0) frame_ok[f] = *reinterpret_cast<const uint32_t*>(fr) == kFrameSync;
}

cudaError_t launch_deframe(const uint8_t* raw, int payload, int64_t f0, int64_t f1, uint8_t* payload_out,
                           uint8_t* frame_ok, cudaStream_t s) {
  if (f1 <= f0) return cudaSuccess;
  const int64_t nf = f1 - f0;
  const int n16 = payload / 16;
  const unsigned gx = (unsigned)((n16 + 255) / 256 < 8 ? (n16 + 255) / 256 : 8);
  const unsigned gy = (unsigned)(nf < 65535 ? nf : 65535);
  const unsigned gz = (unsigned)((nf + gy - 1) / gy);
  k_deframe<<<dim3(gx, gy, gz), 256, 0, s>>>(raw, payload, f0, f1, payload_out, frame_ok);
  return cudaGetLastError();
}

cudaError_t launch_delay_blocks(const DelayParams& p, cudaStream_t s) {
  if (p.nb <= 0) return cudaSuccess;
  dim3 grid((p.nb + 127) / 128, p.S);
  k_delay_blocks<<<grid, 128, 0, s>>>(p);
  return cudaGetLastError();
}

// Debug: codes of stream j of one station for sample-time groups
// [t0, t0 + count) counted from the station's first group (0xFF outside).
__global__ void k_unpack_codes(const StationView* st, int station, int G, int j, int64_t t0,
                               int64_t count, uint8_t* out) {
  const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= count) return;
  const StationView v = st[station];
  const int64_t t = t0 + n;
  uint8_t code = 0xFF;
  if (t >= 0 && t < v.ngroups) {
    const int64_t bit = 2 * (t * G + j);
    const int64_t w = bit >> 5;
    if (w < v.nwords) code = (uint8_t)((v.words[w] >> (bit & 31)) & 3u);
  }
  out[n] = code;
}

cudaError_t launch_unpack_codes(const StationView* st_dev, int station, int G, int j, int64_t t0,
                                int64_t count, uint8_t* out, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  k_unpack_codes<<<(unsigned)((count + 255) / 256), 256, 0, s>>>(st_dev, station, G, j, t0, count, out);
  return cudaGetLastError();
}

}  // namespace corr
