// k_fstage_pre.cu -- the F step with the fringe rotation applied before the
// transform (pre-F).  At a spacecraft's delay rate the fringe phase nu0 tau(t)
// turns several times within one FFT block (the paper, Sec. 2: the dra delay
// model follows RadioAstron's large and fast-changing velocity); one phase per
// block after the transform then averages the fringe away.  Here every
// sample x[n] of a block's window is multiplied by exp(+2 pi i phi_n), with
// phi_n linear about the block centre (phase and rate from the FP64 delay
// model, FP32 increments within the block), the N rotated samples go through
// a complex N-point transform, and channels 0..N/2-1 take the fractional-delay
// slope exp(+2 pi i f_k eps).  Same staging, Stockham passes and store layout
// as the real-transform path (k_fstage_impl.cuh), with L = N points.
#include "k_fstage_impl.cuh"

namespace corr {

cudaError_t fstage_pre_init_constants() { return init_w32(); }

bool fstage_pre_supported(int nchan) { return nchan >= 4 && nchan <= 4096; }

template <int L>
static cudaError_t launch_pre_L(const FParams& p, cudaStream_t st) {
  if constexpr (L >= 256) {
    if (p.G == 16) return launch_LG<L, 16, true>(p, st);
    if (p.G == 32) return launch_LG<L, 32, true>(p, st);
  }
  return launch_LG<L, 0, true>(p, st);
}

cudaError_t launch_fstage_pre(const FParams& p, cudaStream_t s) {
  if (p.CB <= 0) return cudaSuccess;
  switch (2 * p.nchan) {  // N = 2 nchan complex points
    case 8: return launch_pre_L<8>(p, s);
    case 16: return launch_pre_L<16>(p, s);
    case 32: return launch_pre_L<32>(p, s);
    case 64: return launch_pre_L<64>(p, s);
    case 128: return launch_pre_L<128>(p, s);
    case 256: return launch_pre_L<256>(p, s);
    case 512: return launch_pre_L<512>(p, s);
    case 1024: return launch_pre_L<1024>(p, s);
    case 2048: return launch_pre_L<2048>(p, s);
    case 4096: return launch_pre_L<4096>(p, s);
    case 8192: return launch_pre_L<8192>(p, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace corr
