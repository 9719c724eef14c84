// corr_internal.cuh -- shared declarations of the CUDA library (not part of
// the public C ABI).  Kernels: delay blocks (FP64 delay model), the F stage
// (unpack + FFT + rotation), the X stage (cross-multiply-accumulate) and the
// finalisation (weights, normalisation).
#pragma once
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace corr {

// Per-station input stream as seen by the kernels: packed 2-bit samples in
// 32-bit little-endian words; word 0 bit 0 holds stream 0 of station sample
// `sample0`.
struct StationView {
  const uint32_t* words;
  int64_t nwords;    // whole words present
  int64_t sample0;   // station sample index of the first sample-time group
  int64_t ngroups;   // sample-time groups present (for validity)
  int host;          // 1: the words are pinned host memory read over the host link
  // framed input (payload > 0): `words` is the concatenated payload of the
  // frames present; frame_ok[f] says whether frame f carried its sync word
  int payload;              // payload bytes per frame, 0 for plain input
  const uint8_t* frame_ok;  // [nframes]
  int64_t nframes;
};

// Mark5B-style frames: a 16-byte header (word 0 the sync word) and a payload.
constexpr uint32_t kFrameSync = 0xABADDEEDu;
constexpr int kFrameHeader = 16;
// Copy the payloads of frames [f0, f1) of `raw` (frames of 16 + payload bytes)
// to payload[f * payload], and their sync flags to frame_ok[f].
cudaError_t launch_deframe(const uint8_t* raw, int payload, int64_t f0, int64_t f1, uint8_t* payload_out,
                           uint8_t* frame_ok, cudaStream_t s);

constexpr int kMaxStations = 256;
constexpr int kMaxDevices = 64;
constexpr int kMaxSegs = 64;
constexpr int kMaxSub = 64;

// Delay-model inputs for the delay-block kernel.
struct DelayParams {
  int S, nsub, N, G;
  double fs;
  const int* nseg;          // [S]
  const double* seg_t0;     // [S][kMaxSegs]
  const double* seg_c;      // [S][kMaxSegs][6]
  const double* nu0;        // [nsub]
  const StationView* st;    // [S]
  int64_t b0;               // first (absolute) block
  int nb;                   // blocks
  int ld;                   // leading dimension of the outputs (>= nb)
  // outputs, [S][ld] (phi: [S][nsub][ld])
  int64_t* start;           // absolute station sample of the window start
  float* delta;             // eps*fs/N: fractional-delay phase slope, turns per channel
  float* phi;               // frac(nu0*tau), turns
  uint8_t* valid;
  double* eps_out;          // optional (debug): eps in seconds
  double* tau_out;          // optional (debug): tau in seconds
  // optional, pre-F rotation ([S][nsub][ld]): when set, phi holds the phase at
  // the block's first sample instead of its centre, and dphi the phase step
  // per sample in turns as (hi, lo) with hi of at most 10 significant bits
  float2* dphi;
  unsigned long long* max_end;   // optional [S]: max(window end - sample0) over blocks, encoded +2^62
};

// F stage: unpack + real FFT + rotation for CB blocks x S stations x G streams.
struct FParams {
  const StationView* st;    // [S]
  const int64_t* start;     // [S][ld]
  const float* delta;       // [S][ld]
  const float* phi;         // [S][nsub][ld]
  const uint8_t* valid;     // [S][ld]
  const float2* dphi;       // [S][nsub][ld] (pre-F only): phase step per sample, (hi, lo) turns
  int pre;                  // 1: pre-F fringe rotation (phi = phase at the block's first sample)
  int cross;                // 1: spectra in [subband][block][pol][station] order (both hands)
  int ld;
  int blk0;                 // first block of the chunk (index into descriptor arrays)
  int CB;                   // blocks in chunk
  int S, G, npol, nsub, nchan;
  float lut0, lut1, lut2, lut3;
  const float2* twN;        // W_N^m, m < N
  int out_kind;             // 0: complex FP32 spectra; 1: complex FP16 spectra times `scale`;
                            // 2: complex E4M3 spectra times `scale` (Re byte, Im byte)
  float scale;              // exact power of two (FP16 / FP8 output only)
  void* out;                // [G][CB][S][nchan]
};

// MMA operand tiles written by the tensor-core F step: for stream j, channel
// slice sl (W channels), K range kt (64 blocks of FP16, or 128 blocks of FP8)
// two 16 KB tiles (channel groups of cpt), tile index
// ((j * nslice + sl) * NKT + kt) * 2 + group.
struct TcTiles {
  unsigned char* tiles;
  int nslice, NKT, W, cpt;
  int fp8;                  // 0: FP16 tiles (64-block K range); 1: E4M3 tiles (128-block K range)
  float scale;              // exact power of two applied before the FP16 / FP8 rounding
};

// X step on tensor cores from operand tiles (see TcTiles).
struct XTC2Params {
  const unsigned char* tiles;
  int nslice, NKT, S, G, nchan, cpt, W;
  int fp8;                  // tiles hold E4M3 values (MMA kind::f8f6f4) instead of FP16 (kind::f16)
  float2* part;             // [G][nchan][nbl]
  int* err;
  long long wait_limit;     // spins per mbarrier wait (set by the launcher)
};

// X stage: V_ab[k] += X_a[k] conj(X_b[k]) over the chunk's blocks.
struct XParams {
  const float2* spec;       // [G][CB][S][nchan] complex values of kind in_kind
  int in_kind = 0;          // 0: FP32; 1: FP16 (half2); 2: E4M3 pairs (Re low byte) -- S <= 12 only
  int CB, S, G, nchan;
  int KZ;                   // block splits per chunk (one partial each)
  float2* part;             // [KZ][nbl][G][nchan]
  int* err;                 // set to 1 when a device wait times out (may be null)
  long long wait_limit;     // spins per mbarrier wait (set by the launcher)
};

struct FinParams {
  const float2* part;       // [KZ][nbl][G][nchan]
  int KZ, S, G, nchan, N;
  const uint8_t* valid;     // [S][ld]
  int ld, M;                // blocks of the integration
  int* wcount;              // [nbl] scratch
  float2* out;              // [nbl][G][nchan]
  double* weights;          // [nbl] (device, may be null)
  const int* err;           // optional: when *err != 0 (an X-step wait timed out) the output is NaN
  float unscale = 1.0f;     // k_finalize: times this (2^(2 sigma) after an X step on FP16 / E4M3 spectra)
};

// launchers (return cudaError_t of the launch)
cudaError_t launch_delay_blocks(const DelayParams& p, cudaStream_t s);
cudaError_t launch_unpack_codes(const StationView* st_dev, int station, int G, int j, int64_t t0,
                                int64_t count, uint8_t* out, cudaStream_t s);
// Load the F kernels' __constant__ tables into the current device's context
// once (again after a cudaDeviceReset gave the device a new context).
cudaError_t fstage_ensure_constants();
// Id of the CUDA context current on this thread (0 when none is bound or
// the driver cannot say); per-device caches are keyed on it.
unsigned long long current_context_id();
bool fstage_supported(int nchan);
cudaError_t launch_fstage(const FParams& p, cudaStream_t s);
// the pre-F variant (p.pre != 0), nchan <= 4096; launch_fstage dispatches to it
bool fstage_pre_supported(int nchan);
cudaError_t launch_fstage_pre(const FParams& p, cudaStream_t s);
cudaError_t fstage_pre_init_constants();
int xstage_kz(int CB, int S, int G, int nchan);
cudaError_t launch_xstage(const XParams& p, cudaStream_t s);
cudaError_t launch_weights(const FinParams& p, cudaStream_t s);
cudaError_t launch_finalize(const FinParams& p, cudaStream_t s);
// The CUDA-core X step reads FP16 / E4M3 spectra (XParams::in_kind) for up to
// 12 stations and whole 128-channel tiles.
bool xstage_reduced_supported(int S, int nchan);
int xtc_cpt(int S);
// Spins before a device wait of the X kernels gives up (negative: the
// default); process-wide, read at every launch.  A test hook.
void set_wait_limit(long long spins);
long long wait_limit();
bool fstage_tc_tiles_supported(int nchan);
cudaError_t launch_fstage_tc(const FParams& p, const TcTiles& o, cudaStream_t s);
cudaError_t launch_xtc2(const XTC2Params& p, int sm_count, cudaStream_t s);
// FP16 spectra [G][CB][S][nchan] (blocks < cb present) -> operand tiles
cudaError_t launch_tiles(const __half2* spec, const TcTiles& o, int CB, int cb, int S, int G, int nchan,
                         cudaStream_t s);
// E4M3 spectra [G][CB][S][nchan] (two bytes: Re, Im) -> FP8 operand tiles
cudaError_t launch_tiles8(const uint16_t* spec8, const TcTiles& o, int CB, int cb, int S, int G, int nchan,
                          cudaStream_t s);
// finalise for the tensor-core layout [KZ][G][nchan][nbl]; `unscale` undoes the FP16 pre-scale
cudaError_t launch_finalize_tc(const FinParams& p, float unscale, cudaStream_t s);
// finalise of both hands: partials over 2 p.S virtual stations v = pol * S + station and
// p.G = nsub streams (FP32 layout [KZ][nblv][nsub][nchan], or with `tc` the tensor-core
// layout [KZ][nsub][nchan][nblv]); out [nbl][nsub][4][nchan], hand product pq = 2 p + q
cudaError_t launch_finalize_cross(const FinParams& p, bool tc, float unscale, cudaStream_t s);

__host__ __device__ inline int nbl_of(int S) { return S * (S + 1) / 2; }
__host__ __device__ inline int bl_index(int a, int b, int S) { return a * S - a * (a - 1) / 2 + (b - a); }

}  // namespace corr
