// corr_capi.cu -- the handle runtime behind include/corr.h: argument checks,
// station streams in device memory, the delay model on the device, and the
// per-integration schedule of kernels (delay blocks -> [F, X] per chunk ->
// weights -> finalise).
#include "../../include/corr.h"
#include "corr_internal.cuh"

#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

using namespace corr;

constexpr int kStages = 4;  // delay blocks, F, X, weights+finalise
// blocks accumulated in tensor memory (FP32) before the partial sum in HBM

namespace {

thread_local std::string g_create_error;

struct Seg {
  double t0;
  double c[6];
};

struct Station {
  uint8_t* dbuf = nullptr;  // owned device bytes
  size_t cap = 0;
  size_t len = 0;           // bytes present
  const uint8_t* ext = nullptr;  // attached (caller-owned) device bytes
  bool attached = false;
  bool host = false;        // attached bytes live in pinned host memory
  int64_t sample0 = 0;
  bool started = false;     // a push or attach happened
  std::vector<Seg> segs;
  // framed input: the frames' payloads deframed on the device, and their
  // sync flags (frames [0, nframes_done) so far)
  uint8_t* pay = nullptr;
  size_t pay_cap = 0;
  uint8_t* fok = nullptr;
  size_t fok_cap = 0;
  int64_t nframes_done = 0;
  // asynchronous pushes not yet waited for by the compute stream: the byte
  // range of each piece and the event recorded after its copy
  struct Piece {
    size_t start, end;
    cudaEvent_t ev;
  };
  std::vector<Piece> pending;
};

constexpr int kCopyStreams = 2;             // copies alternate between these
constexpr size_t kCopyPiece = (size_t)64 << 20;  // large pushes split into pieces

}  // namespace

struct corr_s {
  int dev = 0;
  int S = 0, nsub = 0, npol = 0, G = 0, nchan = 0, N = 0;
  double tint = 0.0, fs = 32e6;
  int64_t spi = 0;
  float lut[4] = {-3.336f, -1.0f, 1.0f, 3.336f};
  std::vector<double> nu0;
  int precision = CORR_PREC_FP32;
  int rotation = CORR_ROT_POST_F;
  int pol_products = CORR_POL_PARALLEL;
  int payload = 0;  // bytes of payload per Mark5B-style frame, 0: plain packed bytes
  cudaStream_t own_stream = nullptr;
  cudaStream_t copy_stream[kCopyStreams] = {nullptr, nullptr};
  int copy_next = 0;
  cudaStream_t stream = nullptr;
  std::vector<Station> st;
  bool flushed = false;
  int64_t next_int = 0;
  bool polys_dirty = true;
  bool prepared = false;

  // device state
  StationView* d_views = nullptr;
  StationView* h_views = nullptr;  // pinned staging
  bool views_valid = false;        // h_views holds the device copy
  int* d_nseg = nullptr;
  double* d_seg_t0 = nullptr;
  double* d_seg_c = nullptr;
  double* d_nu0 = nullptr;
  int Mcap = 0;
  // Block descriptors, double-buffered: integration i uses slot i & 1, so the
  // next integration's delay blocks are evaluated (on dstream) while this
  // one's F and X steps run.
  int64_t* d_start[2] = {};
  float* d_delta[2] = {};
  float* d_phi[2] = {};
  float2* d_dphi[2] = {};  // pre-F: phase step per sample (hi, lo), [S][nsub][Mcap]
  uint8_t* d_valid[2] = {};
  unsigned long long* d_stat[2] = {};  // [S][3] data-coverage statistics
  unsigned long long* h_stat[2] = {};  // pinned copies
  unsigned long long* h_stat_init = nullptr;  // pinned, the statistics' start values
  float2* d_twN = nullptr;
  int CB = 0, KZ = 0;
  // spectra chunk (and tensor-core tiles): two buffers when the F step of
  // chunk c+1 runs while the X step of chunk c does (on xstream)
  float2* d_spec[2] = {};
  bool overlap = false;
  int pipeline = 1;  // corr_set_pipeline: 1 overlap F and X when the buffers allow, 0 never
  cudaStream_t xstream = nullptr;  // X step, higher priority
  cudaStream_t dstream = nullptr;  // look-ahead delay blocks
  cudaEvent_t ev_f[2] = {}, ev_x[2] = {}, ev_main = nullptr, ev_la = nullptr;
  bool x_pending[2] = {false, false};
  bool la_valid = false;           // integration la_int's delay blocks are (being) evaluated
  int64_t la_int = -1;
  uint64_t model_gen = 1, la_gen = 0;  // bumped whenever the delay model or station data change
  float2* d_part = nullptr;
  float2* d_out = nullptr;
  int* d_wcount = nullptr;
  double* d_wts = nullptr;
  size_t spec_budget = (size_t)1 << 30;
  int chunk_req = 0;  // blocks per F/X chunk requested by the caller (0: from spec_budget)
  int sm_count = 0;
  int sigma = 0;      // FP16 / FP8 spectra carry X * 2^-sigma
  int* d_err = nullptr;
  int* h_err = nullptr;  // pinned
  unsigned char* d_tiles[2] = {};  // tensor-core operand tiles
  bool tc_tiles = false;
  bool tc_direct = false;  // the F step writes the tiles itself
  int x_unit = CORR_X_AUTO;  // requested unit of the X step for FP16 / FP8 spectra
  bool x_cc = false;         // FP16 / FP8 spectra, X step on CUDA cores (FP32 products and sums)

  // optional per-stage CUDA-event timing of the launches
  bool profiling = false;
  struct Mark { int stage; cudaEvent_t a, b; };
  std::vector<Mark> marks;
  std::vector<cudaEvent_t> ev_pool;
  double prof_ms[kStages] = {0};
  int64_t prof_n[kStages] = {0};

  std::string err;

  int fail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    err = buf;
    return code;
  }
  int cuda_fail(cudaError_t e, const char* what) {
    return fail(CORR_ECUDA, "%s: %s", what, cudaGetErrorString(e));
  }
};

#define CK(call, what)                                    \
  do {                                                    \
    cudaError_t e_ = (call);                              \
    if (e_ != cudaSuccess) return h->cuda_fail(e_, what); \
  } while (0)

static bool is_pow2(int x) { return x > 0 && (x & (x - 1)) == 0; }

// The X step's view of the spectra: with both hands of two polarisations it
// runs over 2S virtual stations (station, pol) and nsub streams.
static bool cross_of(const corr_t* h) { return h->pol_products == CORR_POL_CROSS; }
static int x_stations(const corr_t* h) { return cross_of(h) ? 2 * h->S : h->S; }
static int x_streams(const corr_t* h) { return cross_of(h) ? h->nsub : h->G; }
// complex values per baseline in the output: [subband][pol or hand product][channel]
static size_t out_per_baseline(const corr_t* h) {
  return (size_t)h->nsub * (cross_of(h) ? 4 : h->npol) * h->nchan;
}

static int use_device(corr_t* h) {
  int cur = -1;
  cudaGetDevice(&cur);
  if (cur != h->dev) {
    cudaError_t e = cudaSetDevice(h->dev);
    if (e != cudaSuccess) return h->cuda_fail(e, "cudaSetDevice");
  }
  return CORR_OK;
}

static cudaEvent_t take_event(corr_t* h) {
  if (!h->ev_pool.empty()) {
    cudaEvent_t e = h->ev_pool.back();
    h->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}

// Record an event before (begin) / after (end) a stage's launch when profiling.
static cudaEvent_t prof_begin(corr_t* h, cudaStream_t st) {
  if (!h->profiling) return nullptr;
  cudaEvent_t a = take_event(h);
  if (a) cudaEventRecord(a, st);
  return a;
}

static void prof_end(corr_t* h, int stage, cudaEvent_t a, cudaStream_t st) {
  if (!a) return;
  cudaEvent_t b = take_event(h);
  if (!b) {
    h->ev_pool.push_back(a);
    return;
  }
  cudaEventRecord(b, st);
  h->marks.push_back({stage, a, b});
}

// Wait for a look-ahead delay evaluation in flight and forget it.
static int drop_lookahead(corr_t* h) {
  if (h->dstream) {
    cudaError_t e = cudaStreamSynchronize(h->dstream);
    if (e != cudaSuccess) return h->cuda_fail(e, "look-ahead delay blocks");
  }
  h->la_valid = false;
  return CORR_OK;
}

static int prof_collect(corr_t* h) {
  for (auto& m : h->marks) {
    cudaError_t e = cudaEventSynchronize(m.b);
    if (e != cudaSuccess) return h->cuda_fail(e, "profile event");
    float ms = 0.f;
    cudaEventElapsedTime(&ms, m.a, m.b);
    h->prof_ms[m.stage] += ms;
    h->prof_n[m.stage] += 1;
    h->ev_pool.push_back(m.a);
    h->ev_pool.push_back(m.b);
  }
  h->marks.clear();
  return CORR_OK;
}

// All asynchronous copies done (host buffers reusable); compute stream not involved.
static int drain_pushes(corr_t* h) {
  for (int q = 0; q < kCopyStreams; ++q)
    if (h->copy_stream[q]) CK(cudaStreamSynchronize(h->copy_stream[q]), "wait for pushes");
  return CORR_OK;
}

// Whole frames in a station's (framed) bytes.
static int64_t station_frames(const corr_t* h, const Station& s) {
  return h->payload > 0 ? (int64_t)(s.len / (size_t)(kFrameHeader + h->payload)) : 0;
}

// Sample-time groups a station's bytes hold (for framed input: those of the
// whole frames' payloads).
static int64_t station_groups(const corr_t* h, const Station& s) {
  const size_t bytes = h->payload > 0 ? (size_t)station_frames(h, s) * h->payload : s.len;
  return (int64_t)((bytes * 4) / (size_t)h->G);
}

static const uint8_t* station_ptr(const Station& s) { return s.attached ? s.ext : s.dbuf; }

static int64_t integ_first_block(const corr_t* h, int64_t i) {
  return (i * h->spi + h->N - 1) / h->N;
}

// ------------------------------------------------------------------------
// device preparation

static void free_device(corr_t* h) {
  cudaFree(h->d_views);
  cudaFreeHost(h->h_views);
  cudaFree(h->d_nseg);
  cudaFree(h->d_seg_t0);
  cudaFree(h->d_seg_c);
  cudaFree(h->d_nu0);
  for (int q = 0; q < 2; ++q) {
    cudaFree(h->d_start[q]);
    cudaFree(h->d_delta[q]);
    cudaFree(h->d_phi[q]);
    cudaFree(h->d_dphi[q]);
    cudaFree(h->d_valid[q]);
    cudaFree(h->d_stat[q]);
    cudaFreeHost(h->h_stat[q]);
    cudaFree(h->d_spec[q]);
    cudaFree(h->d_tiles[q]);
    h->d_start[q] = nullptr; h->d_delta[q] = nullptr; h->d_phi[q] = nullptr; h->d_dphi[q] = nullptr;
    h->d_valid[q] = nullptr; h->d_stat[q] = nullptr; h->h_stat[q] = nullptr; h->d_spec[q] = nullptr;
    h->d_tiles[q] = nullptr;
    if (h->ev_f[q]) cudaEventDestroy(h->ev_f[q]);
    if (h->ev_x[q]) cudaEventDestroy(h->ev_x[q]);
    h->ev_f[q] = h->ev_x[q] = nullptr;
    h->x_pending[q] = false;
  }
  if (h->ev_main) cudaEventDestroy(h->ev_main);
  if (h->ev_la) cudaEventDestroy(h->ev_la);
  h->ev_main = h->ev_la = nullptr;
  cudaFreeHost(h->h_stat_init);
  h->h_stat_init = nullptr;
  cudaFree(h->d_twN);
  cudaFree(h->d_part);
  cudaFree(h->d_out);
  cudaFree(h->d_wcount);
  cudaFree(h->d_wts);
  h->d_wts = nullptr;
  cudaFree(h->d_err);
  cudaFreeHost(h->h_err);
  h->d_err = nullptr;
  h->h_err = nullptr;
  h->d_views = nullptr; h->h_views = nullptr; h->d_nseg = nullptr; h->d_seg_t0 = nullptr;
  h->d_seg_c = nullptr; h->d_nu0 = nullptr;
  h->d_twN = nullptr; h->d_part = nullptr; h->d_out = nullptr;
  h->d_wcount = nullptr;
  h->prepared = false;
  h->views_valid = false;
  h->la_valid = false;
}

static int dalloc(corr_t* h, void** p, size_t bytes, const char* what) {
  cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return h->fail(CORR_ENOMEM, "cudaMalloc %s (%zu bytes): %s", what, bytes, cudaGetErrorString(e));
  }
  return CORR_OK;
}

// Sizes of the work buffers, from the handle's shape alone (shared by the
// allocation and by the memory estimate a scheduler asks for).
struct WorkLayout {
  int64_t spi = 0;
  int Mcap = 0, CB = 0, KZ = 0;
  bool tiles = false, direct = false;
  bool cc = false;  // FP16 / FP8 spectra read by the CUDA-core X step
  int nbuf = 1;  // spectra / tile buffers: 2 when F and X overlap
  size_t spec = 0, part = 0, tiles_bytes = 0, small = 0;  // spec, tiles_bytes: per buffer
  size_t total() const { return nbuf * (spec + tiles_bytes) + part + small; }
};

// F and X overlap (two spectra / tile buffers) unless one buffer is already
// this large: the dense many-station shapes, which the F step dominates.
constexpr size_t kOverlapMaxBuffer = (size_t)4 << 30;

static int work_layout(corr_t* h, WorkLayout& w) {
  const double spi = h->fs * h->tint;
  if (fabs(spi - (double)llround(spi)) > 1e-6 || llround(spi) < h->N)
    return h->fail(CORR_EINVAL, "fs*tint = %.9g must be a whole number of samples >= 2*nchan", spi);
  w.spi = llround(spi);
  const int S = h->S, G = h->G, nch = h->nchan;
  const int XS = x_stations(h), XG = x_streams(h);
  const size_t nbl = (size_t)nbl_of(S);
  w.Mcap = (int)((w.spi + h->N - 1) / h->N) + 1;
  const size_t per_block = (size_t)G * S * nch * sizeof(float2);
  const bool fp8 = h->precision == CORR_PREC_FP8_TC;
  // FP16 / FP8 spectra: the X step on the tensor cores, or (up to 12
  // (station, pol) rows, where an MMA tile would be mostly padding and the
  // operand corner turn costs more than the X step it speeds up) on the
  // CUDA cores from the same spectra
  w.cc = h->precision != CORR_PREC_FP32 && h->x_unit != CORR_X_TENSOR_CORES &&
         xstage_reduced_supported(XS, nch) && (h->x_unit == CORR_X_CUDA_CORES || XS <= 12);
  const bool tc = h->precision != CORR_PREC_FP32 && !w.cc;
  const int kb = fp8 ? 128 : 64;  // blocks per K tile
  // the F step writes tensor-core tiles itself for FFTs of up to 2048 points
  // and post-F rotation; otherwise FP16 / FP8 spectra are corner-turned
  const bool direct_ok = fstage_tc_tiles_supported(nch) && h->rotation == CORR_ROT_POST_F && !cross_of(h);
  int64_t cb = h->chunk_req > 0 ? h->chunk_req : (int64_t)(h->spec_budget / per_block);
  if (h->chunk_req <= 0) {
    // Every chunk reads and writes all partial visibilities once; chunks of at
    // least 32 (S + 1) / b blocks (b = bytes per complex spectrum value) keep
    // that traffic near a quarter of the spectra the X step reads.  On the
    // tensor cores a chunk of 512 blocks also gives each accumulator 8 K tiles
    // before its read-out.  Up to four times the FP32 spectra budget is spent
    // on it; the tensor cores count what they hold per block (operand tiles,
    // plus FP16 / FP8 spectra when a corner turn builds the tiles) against
    // sixteen times the budget, since at many stations every accumulator
    // read-out costs as much as several K tiles.
    const int64_t want = tc ? std::max<int64_t>(8 * (int64_t)(XS + 1), 512) : 4 * (int64_t)(XS + 1);
    int64_t cap = (int64_t)(4 * h->spec_budget / per_block);
    if (tc && xtc_cpt(XS) > 0) {
      const int W = 2 * xtc_cpt(XS);
      const size_t tiles_per_block = (size_t)XG * ((nch + W - 1) / W) * 32768 / kb;
      const size_t tc_per_block = tiles_per_block + (direct_ok ? 0 : per_block / (fp8 ? 4 : 2));
      cap = std::max<int64_t>(cap, (int64_t)(16 * h->spec_budget / tc_per_block));
    }
    if (cb < want) cb = std::min(want, std::max(cap, cb));
  }
  if (cb < 1) cb = 1;
  if (cb > w.Mcap) cb = w.Mcap;
  // the tensor cores read whole K tiles: a default chunk of whole tiles leaves
  // no zero padding except in the last chunk of an integration
  if (tc && h->chunk_req <= 0 && cb > kb) cb -= cb % kb;
  w.CB = (int)cb;
  w.KZ = xstage_kz(w.CB, XS, XG, nch);
  // tensor-core operand tiles hold up to 64 stations; for FFTs of up to 2048
  // points the F step writes them directly, above that FP16 (FP8) spectra are
  // corner-turned into them
  w.tiles = tc && xtc_cpt(XS) > 0;
  w.direct = w.tiles && direct_ok;
  w.spec = w.direct ? 16
                    : ((w.tiles || w.cc) ? per_block / (fp8 ? 4 : 2) * w.CB : per_block * w.CB);
  // partial sums: KZ slices for the FP32 X step, one for the tensor cores
  w.part = sizeof(float2) * (size_t)(tc ? 1 : w.KZ) * nbl_of(XS) * XG * nch;
  if (w.tiles) {
    const int W = 2 * xtc_cpt(XS);
    w.tiles_bytes = (size_t)XG * ((nch + W - 1) / W) * ((size_t)(w.CB + kb - 1) / kb) * 32768;
  }
  w.nbuf = (h->pipeline && w.spec + w.tiles_bytes <= kOverlapMaxBuffer) ? 2 : 1;
  const size_t M = (size_t)w.Mcap;
  // descriptors (two slots), model, twiddles, output, weights
  w.small = sizeof(StationView) * S + sizeof(int) * S + sizeof(double) * S * kMaxSegs * 7 +
            sizeof(double) * h->nsub +
            2 * ((sizeof(int64_t) + sizeof(float) + 1) * S * M + sizeof(float) * S * h->nsub * M +
                 sizeof(unsigned long long) * 3 * S +
                 (h->rotation == CORR_ROT_PRE_F ? sizeof(float2) * S * h->nsub * M : 0)) +
            sizeof(float2) * h->N + sizeof(float2) * nbl * out_per_baseline(h) + (sizeof(int) + sizeof(double)) * nbl +
            sizeof(int);
  return CORR_OK;
}

static int prepare(corr_t* h) {
  if (h->prepared) return CORR_OK;
  WorkLayout w;
  int rc;
  if ((rc = work_layout(h, w))) return rc;
  h->spi = w.spi;
  CK(fstage_ensure_constants(), "fstage constants");
  const int S = h->S, G = h->G, nch = h->nchan, nbl = nbl_of(S);
  h->Mcap = w.Mcap;
  h->CB = w.CB;
  h->KZ = w.KZ;
  {
    // FP16: 2^-floor(log2(N)/2) keeps |X| <= 3.336 N far inside the FP16
    // range; FP8 (E4M3, largest value 448): four times larger, which puts the
    // RMS of a component of X (about 1.47 sqrt(N) for 2-bit noise) near 8
    int lg = 0;
    while ((1 << (lg + 1)) <= h->N) ++lg;
    h->sigma = lg / 2 - (h->precision == CORR_PREC_FP8_TC ? 2 : 0);
  }
  CK(cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, h->dev), "SM count");
  if ((rc = dalloc(h, (void**)&h->d_views, sizeof(StationView) * S, "views"))) return rc;
  CK(cudaMallocHost((void**)&h->h_views, sizeof(StationView) * S), "cudaMallocHost views");
  if ((rc = dalloc(h, (void**)&h->d_nseg, sizeof(int) * S, "nseg"))) return rc;
  if ((rc = dalloc(h, (void**)&h->d_seg_t0, sizeof(double) * S * kMaxSegs, "seg_t0"))) return rc;
  if ((rc = dalloc(h, (void**)&h->d_seg_c, sizeof(double) * S * kMaxSegs * 6, "seg_c"))) return rc;
  if ((rc = dalloc(h, (void**)&h->d_nu0, sizeof(double) * h->nsub, "nu0"))) return rc;
  for (int q = 0; q < 2; ++q) {
    if ((rc = dalloc(h, (void**)&h->d_start[q], sizeof(int64_t) * S * h->Mcap, "start"))) return rc;
    if ((rc = dalloc(h, (void**)&h->d_delta[q], sizeof(float) * S * h->Mcap, "delta"))) return rc;
    if ((rc = dalloc(h, (void**)&h->d_phi[q], sizeof(float) * S * h->nsub * h->Mcap, "phi"))) return rc;
    if (h->rotation == CORR_ROT_PRE_F &&
        (rc = dalloc(h, (void**)&h->d_dphi[q], sizeof(float2) * S * h->nsub * h->Mcap, "phase steps")))
      return rc;
    if ((rc = dalloc(h, (void**)&h->d_valid[q], (size_t)S * h->Mcap, "valid"))) return rc;
    if ((rc = dalloc(h, (void**)&h->d_stat[q], sizeof(unsigned long long) * 3 * S, "stat"))) return rc;
    CK(cudaMallocHost((void**)&h->h_stat[q], sizeof(unsigned long long) * 3 * S), "cudaMallocHost stat");
  }
  CK(cudaMallocHost((void**)&h->h_stat_init, sizeof(unsigned long long) * 3 * S), "cudaMallocHost stat");
  for (int s = 0; s < S; ++s) {
    h->h_stat_init[3 * s + 0] = 0ull;   // max window end
    h->h_stat_init[3 * s + 1] = ~0ull;  // min window start
    h->h_stat_init[3 * s + 2] = 0ull;   // valid blocks
  }
  if ((rc = dalloc(h, (void**)&h->d_twN, sizeof(float2) * h->N, "twiddles"))) return rc;
  h->overlap = w.nbuf == 2;
  for (int q = 0; q < w.nbuf; ++q)
    if ((rc = dalloc(h, (void**)&h->d_spec[q], w.spec, "spectra"))) return rc;
  for (int q = 0; q < 2; ++q) {
    CK(cudaEventCreateWithFlags(&h->ev_f[q], cudaEventDisableTiming), "events");
    CK(cudaEventCreateWithFlags(&h->ev_x[q], cudaEventDisableTiming), "events");
  }
  CK(cudaEventCreateWithFlags(&h->ev_main, cudaEventDisableTiming), "events");
  CK(cudaEventCreateWithFlags(&h->ev_la, cudaEventDisableTiming), "events");
  if ((rc = dalloc(h, (void**)&h->d_part, w.part, "partials"))) return rc;
  if ((rc = dalloc(h, (void**)&h->d_out, sizeof(float2) * (size_t)nbl * out_per_baseline(h), "out"))) return rc;
  if ((rc = dalloc(h, (void**)&h->d_wcount, sizeof(int) * nbl, "wcount"))) return rc;
  if ((rc = dalloc(h, (void**)&h->d_wts, sizeof(double) * nbl, "weights"))) return rc;
  if ((rc = dalloc(h, (void**)&h->d_err, sizeof(int), "error flag"))) return rc;
  CK(cudaMallocHost((void**)&h->h_err, sizeof(int)), "cudaMallocHost err");
  h->tc_tiles = w.tiles;
  h->tc_direct = w.direct;
  h->x_cc = w.cc;
  if (h->tc_tiles) {
    for (int q = 0; q < w.nbuf; ++q) {
      if ((rc = dalloc(h, (void**)&h->d_tiles[q], w.tiles_bytes, "operand tiles"))) return rc;
      // rows beyond the stations of a tile stay zero for good
      CK(cudaMemset(h->d_tiles[q], 0, w.tiles_bytes), "operand tiles clear");
    }
  }
  *h->h_err = 0;
  CK(cudaMemset(h->d_err, 0, sizeof(int)), "error flag reset");
  // W_N^m = exp(-2 pi i m / N), computed in FP64 on the host
  std::vector<float2> tw(h->N);
  for (int m = 0; m < h->N; ++m) {
    double a = -2.0 * 3.14159265358979323846 * (double)m / (double)h->N;
    tw[m] = make_float2((float)cos(a), (float)sin(a));
  }
  CK(cudaMemcpy(h->d_twN, tw.data(), sizeof(float2) * h->N, cudaMemcpyHostToDevice), "twiddles H2D");
  h->prepared = true;
  h->polys_dirty = true;
  return CORR_OK;
}

// Deframe every station's frames that arrived since the last call into its
// payload buffer (grown as needed), with their sync flags.
static int deframe_new(corr_t* h) {
  for (Station& x : h->st) {
    const int64_t nf = station_frames(h, x);
    if (nf <= x.nframes_done) continue;
    if (!x.pending.empty()) {  // asynchronous pushes: the frames must have landed
      int rc = drain_pushes(h);
      if (rc) return rc;
    }
    const size_t need_pay = (size_t)nf * h->payload, need_ok = (size_t)nf;
    if (need_pay > x.pay_cap || need_ok > x.fok_cap) {
      // the F step and a look-ahead delay evaluation may still read the old buffers
      int rc = drop_lookahead(h);
      if (rc) return rc;
      CK(cudaStreamSynchronize(h->stream), "sync before payload growth");
      size_t cp = x.pay_cap ? x.pay_cap : ((size_t)1 << 20);
      while (cp < need_pay) cp *= 2;
      size_t co = x.fok_cap ? x.fok_cap : 4096;
      while (co < need_ok) co *= 2;
      uint8_t *np = nullptr, *no = nullptr;
      if ((rc = dalloc(h, (void**)&np, cp, "frame payloads"))) return rc;
      if ((rc = dalloc(h, (void**)&no, co, "frame flags"))) {
        cudaFree(np);
        return rc;
      }
      const size_t done_pay = (size_t)x.nframes_done * h->payload;
      cudaError_t e = cudaSuccess;
      if (done_pay) e = cudaMemcpyAsync(np, x.pay, done_pay, cudaMemcpyDeviceToDevice, h->stream);
      if (e == cudaSuccess && x.nframes_done)
        e = cudaMemcpyAsync(no, x.fok, (size_t)x.nframes_done, cudaMemcpyDeviceToDevice, h->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
      if (e != cudaSuccess) {
        cudaFree(np);
        cudaFree(no);
        return h->cuda_fail(e, "payload growth");
      }
      cudaFree(x.pay);
      cudaFree(x.fok);
      x.pay = np;
      x.pay_cap = cp;
      x.fok = no;
      x.fok_cap = co;
    }
    CK(launch_deframe(station_ptr(x), h->payload, x.nframes_done, nf, x.pay, x.fok, h->stream), "deframe launch");
    x.nframes_done = nf;
  }
  return CORR_OK;
}

static int upload_model(corr_t* h) {
  const int S = h->S;
  for (int s = 0; s < S; ++s)
    if (h->st[s].segs.empty()) return h->fail(CORR_EINVAL, "station %d has no delay polynomial", s);
  if (h->polys_dirty) {
    // a look-ahead delay evaluation may still read the old model
    int rc0 = drop_lookahead(h);
    if (rc0) return rc0;
    h->model_gen += 1;
    std::vector<int> nseg(S);
    std::vector<double> t0((size_t)S * kMaxSegs, 0.0), c((size_t)S * kMaxSegs * 6, 0.0);
    for (int s = 0; s < S; ++s) {
      nseg[s] = (int)h->st[s].segs.size();
      for (int q = 0; q < nseg[s]; ++q) {
        t0[(size_t)s * kMaxSegs + q] = h->st[s].segs[q].t0;
        memcpy(&c[((size_t)s * kMaxSegs + q) * 6], h->st[s].segs[q].c, sizeof(double) * 6);
      }
    }
    CK(cudaMemcpy(h->d_nseg, nseg.data(), sizeof(int) * S, cudaMemcpyHostToDevice), "nseg H2D");
    CK(cudaMemcpy(h->d_seg_t0, t0.data(), sizeof(double) * t0.size(), cudaMemcpyHostToDevice), "t0 H2D");
    CK(cudaMemcpy(h->d_seg_c, c.data(), sizeof(double) * c.size(), cudaMemcpyHostToDevice), "coeff H2D");
    CK(cudaMemcpy(h->d_nu0, h->nu0.data(), sizeof(double) * h->nsub, cudaMemcpyHostToDevice), "nu0 H2D");
    h->polys_dirty = false;
  }
  // framed input: deframe the frames that arrived since the last call
  if (h->payload > 0) {
    int rc2 = deframe_new(h);
    if (rc2) return rc2;
  }
  // station views: the pinned staging copy holds what the device has; copy
  // again only when a push or attach changed them
  std::vector<StationView> views(S);
  for (int s = 0; s < S; ++s) {
    const Station& x = h->st[s];
    StationView& v = views[s];
    memset(&v, 0, sizeof(v));
    v.words = reinterpret_cast<const uint32_t*>(station_ptr(x));
    v.host = x.host ? 1 : 0;
    v.nwords = (int64_t)(x.len / 4);
    v.sample0 = x.sample0;
    v.ngroups = station_groups(h, x);
    if (h->payload > 0) {  // the kernels read the deframed payload (device memory)
      v.words = reinterpret_cast<const uint32_t*>(x.pay);
      v.host = 0;
      v.nwords = x.nframes_done * (int64_t)h->payload / 4;
      v.payload = h->payload;
      v.frame_ok = x.fok;
      v.nframes = x.nframes_done;
    }
  }
  if (h->views_valid && memcmp(views.data(), h->h_views, sizeof(StationView) * S) == 0) return CORR_OK;
  // the F step and a look-ahead delay evaluation may still read the old views
  int rc1 = drop_lookahead(h);
  if (rc1) return rc1;
  h->model_gen += 1;
  CK(cudaStreamSynchronize(h->stream), "sync before view update");
  memcpy(h->h_views, views.data(), sizeof(StationView) * S);
  CK(cudaMemcpyAsync(h->d_views, h->h_views, sizeof(StationView) * S, cudaMemcpyHostToDevice, h->stream),
     "views H2D");
  h->views_valid = true;
  return CORR_OK;
}

static DelayParams delay_params(corr_t* h, int64_t b0, int nb, int ld, int slot) {
  DelayParams p;
  p.S = h->S;
  p.nsub = h->nsub;
  p.N = h->N;
  p.G = h->G;
  p.fs = h->fs;
  p.nseg = h->d_nseg;
  p.seg_t0 = h->d_seg_t0;
  p.seg_c = h->d_seg_c;
  p.nu0 = h->d_nu0;
  p.st = h->d_views;
  p.b0 = b0;
  p.nb = nb;
  p.ld = ld;
  p.start = h->d_start[slot];
  p.delta = h->d_delta[slot];
  p.phi = h->d_phi[slot];
  p.valid = h->d_valid[slot];
  p.eps_out = nullptr;
  p.tau_out = nullptr;
  p.max_end = nullptr;
  p.dphi = h->d_dphi[slot];  // null unless pre-F
  return p;
}

static FParams fparams(corr_t* h, int blk0, int cb, int slot) {
  FParams p;
  p.st = h->d_views;
  p.start = h->d_start[slot];
  p.delta = h->d_delta[slot];
  p.phi = h->d_phi[slot];
  p.valid = h->d_valid[slot];
  p.dphi = h->d_dphi[slot];
  p.pre = h->rotation == CORR_ROT_PRE_F ? 1 : 0;
  p.cross = cross_of(h) ? 1 : 0;
  p.ld = h->Mcap;
  p.blk0 = blk0;
  p.CB = cb;
  p.S = h->S;
  p.G = h->G;
  p.npol = h->npol;
  p.nsub = h->nsub;
  p.nchan = h->nchan;
  p.lut0 = h->lut[0];
  p.lut1 = h->lut[1];
  p.lut2 = h->lut[2];
  p.lut3 = h->lut[3];
  p.twN = h->d_twN;
  p.out_kind = 0;
  p.scale = 1.0f;
  p.out = h->d_spec[0];
  return p;
}

// Device work of one integration after its delay blocks are in descriptor
// slot `slot`: partial-sum clear, F and X per chunk, weights and
// normalisation, with no host wait (so it can be recorded into a CUDA graph).
// M = blocks of the integration.  With `overlap` the X step of each chunk
// runs on xstream while the F step of the next chunk runs on st (two
// spectra / tile buffers, events between them); everything joins st again
// before the weights.  Without it every launch goes to st.
static int enqueue_rest(corr_t* h, cudaStream_t st, int M, float2* vis_out, double* w_out, int slot, bool overlap) {
  const int S = h->S;
  cudaEvent_t pa = nullptr;
  const bool reduced = h->precision != CORR_PREC_FP32;  // FP16 / FP8 spectra
  const bool fp8 = h->precision == CORR_PREC_FP8_TC;
  const bool tc = h->tc_tiles;                           // X step on the tensor cores
  const int kz_used = tc ? 1 : h->KZ;
  // the X step's stations and streams (2S and nsub with both hands)
  const int XS = x_stations(h), XG = x_streams(h);
  cudaStream_t xs = overlap ? h->xstream : st;
  CK(cudaMemsetAsync(h->d_part, 0, sizeof(float2) * (size_t)kz_used * nbl_of(XS) * XG * h->nchan, st),
     "partials memset");
  int c = 0;
  for (int c0 = 0; c0 < M; c0 += h->CB, ++c) {
    const int buf = overlap ? (c & 1) : 0;
    const int cb = (M - c0 < h->CB) ? (M - c0) : h->CB;
    // the F step writes buffer `buf`: the X step that read it last must be done
    if (overlap && h->x_pending[buf]) {
      CK(cudaStreamWaitEvent(st, h->ev_x[buf], 0), "wait for the X step");
      h->x_pending[buf] = false;
    }
    FParams fp = fparams(h, c0, cb, slot);
    fp.out = h->d_spec[buf];
    if (reduced) {
      fp.out_kind = fp8 ? 2 : 1;
      fp.scale = ldexpf(1.0f, -h->sigma);
    }
    if (h->tc_tiles) {
      // MMA operand tiles, fetched by the X step with bulk copies: written by
      // the F step itself, or corner-turned from FP16 / FP8 spectra
      TcTiles o;
      o.tiles = h->d_tiles[buf];
      o.cpt = xtc_cpt(XS);
      o.W = 2 * o.cpt;
      o.nslice = (h->nchan + o.W - 1) / o.W;
      o.fp8 = fp8 ? 1 : 0;
      o.NKT = fp8 ? (cb + 127) / 128 : (cb + 63) / 64;
      o.scale = ldexpf(1.0f, -h->sigma);
      pa = prof_begin(h, st);
      if (h->tc_direct) {
        CK(launch_fstage_tc(fp, o, st), "tensor-core fstage launch");
      } else {
        CK(launch_fstage(fp, st), "fstage launch");
        if (fp8)
          CK(launch_tiles8(reinterpret_cast<const uint16_t*>(h->d_spec[buf]), o, cb, cb, XS, XG, h->nchan, st),
             "FP8 tile corner-turn launch");
        else
          CK(launch_tiles(reinterpret_cast<const __half2*>(h->d_spec[buf]), o, cb, cb, XS, XG, h->nchan, st),
             "tile corner-turn launch");
      }
      prof_end(h, 1, pa, st);
      if (overlap) {
        CK(cudaEventRecord(h->ev_f[buf], st), "F event");
        CK(cudaStreamWaitEvent(xs, h->ev_f[buf], 0), "wait for the F step");
      }
      XTC2Params xp;
      xp.tiles = h->d_tiles[buf];
      xp.nslice = o.nslice;
      xp.NKT = o.NKT;
      xp.S = XS;
      xp.G = XG;
      xp.nchan = h->nchan;
      xp.cpt = o.cpt;
      xp.W = o.W;
      xp.fp8 = o.fp8;
      xp.part = h->d_part;
      xp.err = h->d_err;
      pa = prof_begin(h, xs);
      CK(launch_xtc2(xp, h->sm_count, xs), "tensor-core xstage launch");
      prof_end(h, 2, pa, xs);
    } else {
      pa = prof_begin(h, st);
      CK(launch_fstage(fp, st), "fstage launch");
      prof_end(h, 1, pa, st);
      if (overlap) {
        CK(cudaEventRecord(h->ev_f[buf], st), "F event");
        CK(cudaStreamWaitEvent(xs, h->ev_f[buf], 0), "wait for the F step");
      }
      XParams xp;
      xp.spec = h->d_spec[buf];
      xp.in_kind = h->x_cc ? (fp8 ? 2 : 1) : 0;
      xp.CB = cb;
      xp.S = XS;
      xp.G = XG;
      xp.nchan = h->nchan;
      xp.KZ = h->KZ;
      xp.part = h->d_part;
      xp.err = h->d_err;
      pa = prof_begin(h, xs);
      CK(launch_xstage(xp, xs), "xstage launch");
      prof_end(h, 2, pa, xs);
    }
    if (overlap) {
      CK(cudaEventRecord(h->ev_x[buf], xs), "X event");
      h->x_pending[buf] = true;
    }
  }
  // every X step of the integration before the weights and normalisation
  for (int q = 0; q < 2; ++q)
    if (h->x_pending[q]) {
      CK(cudaStreamWaitEvent(st, h->ev_x[q], 0), "wait for the X step");
      h->x_pending[q] = false;
    }
  FinParams fin;
  fin.part = h->d_part;
  fin.KZ = kz_used;
  fin.S = S;
  fin.G = h->G;
  fin.nchan = h->nchan;
  fin.N = h->N;
  fin.valid = h->d_valid[slot];
  fin.ld = h->Mcap;
  fin.M = M;
  fin.wcount = h->d_wcount;
  fin.out = vis_out;
  fin.weights = w_out;
  fin.err = nullptr;  // the handle reports a device timeout as CORR_ETIMEOUT
  pa = prof_begin(h, st);
  CK(launch_weights(fin, st), "weights launch");
  // FP16 / FP8 spectra carry X 2^-sigma: the sums carry 2^(-2 sigma)
  const float unscale = reduced ? ldexpf(1.0f, 2 * h->sigma) : 1.0f;
  if (cross_of(h)) {
    fin.G = h->nsub;
    CK(launch_finalize_cross(fin, tc, unscale, st), "finalize launch");
  } else if (tc) {
    CK(launch_finalize_tc(fin, unscale, st), "finalize launch");
  } else {
    fin.unscale = unscale;
    CK(launch_finalize(fin, st), "finalize launch");
  }
  prof_end(h, 3, pa, st);
  return CORR_OK;
}

// Delay blocks of integration i into descriptor slot i & 1 on stream st,
// with the data-coverage statistics copied to the slot's pinned host copy.
static int enqueue_delays(corr_t* h, int64_t i, cudaStream_t st) {
  const int S = h->S;
  const int slot = (int)(i & 1);
  const int64_t bfirst = integ_first_block(h, i);
  const int M = (int)(integ_first_block(h, i + 1) - bfirst);
  CK(cudaMemcpyAsync(h->d_stat[slot], h->h_stat_init, sizeof(unsigned long long) * 3 * S, cudaMemcpyHostToDevice, st),
     "stat H2D");
  DelayParams dp = delay_params(h, bfirst, M, h->Mcap, slot);
  dp.max_end = h->d_stat[slot];
  cudaEvent_t pa = prof_begin(h, st);
  CK(launch_delay_blocks(dp, st), "delay_blocks launch");
  prof_end(h, 0, pa, st);
  CK(cudaMemcpyAsync(h->h_stat[slot], h->d_stat[slot], sizeof(unsigned long long) * 3 * S, cudaMemcpyDeviceToHost, st),
     "stat D2H");
  return CORR_OK;
}

// The whole schedule of one integration.  On success the visibilities are in
// vis_out (device, [nbl][G][nchan]) and, if given, the weights in w_out.
static int run_integration(corr_t* h, float2* vis_out, double* w_out) {
  int rc;
  if ((rc = use_device(h))) return rc;
  if ((rc = prepare(h))) return rc;
  if ((rc = upload_model(h))) return rc;
  const int S = h->S;
  const int64_t i = h->next_int;
  const int slot = (int)(i & 1);
  const int64_t bfirst = integ_first_block(h, i);
  const int M = (int)(integ_first_block(h, i + 1) - bfirst);

  // 1. delay blocks + data-coverage statistics: evaluated ahead during the
  //    previous integration (for the same model and data), or now
  if (h->la_valid && h->la_int == i && h->la_gen == h->model_gen) {
    CK(cudaEventSynchronize(h->ev_la), "look-ahead delay blocks");
    CK(cudaStreamWaitEvent(h->stream, h->ev_la, 0), "wait for the delay blocks");
    h->la_valid = false;
  } else {
    if ((rc = drop_lookahead(h))) return rc;
    if ((rc = enqueue_delays(h, i, h->stream))) return rc;
    CK(cudaStreamSynchronize(h->stream), "delay_blocks");
  }
  if (*h->h_err) return h->fail(CORR_ETIMEOUT, "an X-step wait timed out on the device");
  const unsigned long long off = 1ull << 62;
  const unsigned long long* stat = h->h_stat[slot];
  // the compute stream waits for the asynchronous pushes holding the bytes
  // this integration reads (pieces that start below the last byte needed)
  for (int s = 0; s < S; ++s) {
    Station& x = h->st[s];
    if (x.pending.empty()) continue;
    const int64_t need = (int64_t)(stat[3 * s + 0] - off);
    const size_t need_bytes = need > 0 ? (size_t)((need * (int64_t)h->G * 2 + 7) / 8) : 0;
    size_t keep = 0;
    for (size_t q = 0; q < x.pending.size(); ++q) {
      if (x.pending[q].start < need_bytes || h->flushed) {
        CK(cudaStreamWaitEvent(h->stream, x.pending[q].ev, 0), "wait for pushed samples");
        cudaEventDestroy(x.pending[q].ev);
      } else {
        x.pending[keep++] = x.pending[q];
      }
    }
    x.pending.resize(keep);
  }
  bool any_data = false;
  for (int s = 0; s < S; ++s) {
    const int64_t need = (int64_t)(stat[3 * s + 0] - off);
    const int64_t first = (int64_t)(stat[3 * s + 1] - off);
    const int64_t have = station_groups(h, h->st[s]);
    if (need > have && !h->flushed)
      return h->fail(CORR_EAGAIN, "station %d: integration %lld needs %lld sample groups, %lld present", s,
                     (long long)i, (long long)need, (long long)have);
    if (first + h->N <= have) any_data = true;
  }
  if (h->flushed && !any_data) return h->fail(CORR_EEND, "no station has data for integration %lld", (long long)i);

  // the other descriptor slot is free once everything enqueued so far
  // (integration i-1's F and weights) has run
  CK(cudaEventRecord(h->ev_main, h->stream), "main event");
  int rc2 = enqueue_rest(h, h->stream, M, vis_out, w_out, slot, h->overlap);
  if (rc2) return rc2;
  CK(cudaMemcpyAsync(h->h_err, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, h->stream), "error flag D2H");
  h->next_int = i + 1;
  // 2. look-ahead: the next integration's delay blocks, on their own stream,
  //    while this integration's F and X steps run
  CK(cudaStreamWaitEvent(h->dstream, h->ev_main, 0), "look-ahead wait");
  if ((rc = enqueue_delays(h, i + 1, h->dstream))) return rc;
  CK(cudaEventRecord(h->ev_la, h->dstream), "look-ahead event");
  h->la_valid = true;
  h->la_int = i + 1;
  h->la_gen = h->model_gen;
  return CORR_OK;
}

// ------------------------------------------------------------------------
// C ABI

extern "C" {

int corr_create(corr_t** hp, int stations, int subbands, int pols, int nchan, double tint_s) {
  if (!hp) {
    g_create_error = "corr_create: h is NULL";
    return CORR_EINVAL;
  }
  *hp = nullptr;
  if (stations < 1 || stations > kMaxStations) {
    g_create_error = "corr_create: stations must be 1..256";
    return CORR_EINVAL;
  }
  if (pols < 1 || pols > 2 || subbands < 1 || subbands * pols > 32 || subbands > kMaxSub) {
    g_create_error = "corr_create: need pols 1..2 and 1 <= subbands*pols <= 32";
    return CORR_EINVAL;
  }
  if (!is_pow2(nchan) || nchan < 4 || nchan > 8192 || !fstage_supported(nchan)) {
    g_create_error = "corr_create: nchan must be a power of two in 4..8192";
    return CORR_EINVAL;
  }
  if (!(tint_s > 0.0) || !isfinite(tint_s)) {
    g_create_error = "corr_create: tint must be > 0";
    return CORR_EINVAL;
  }
  corr_t* h = new (std::nothrow) corr_t();
  if (!h) {
    g_create_error = "corr_create: out of host memory";
    return CORR_ENOMEM;
  }
  h->S = stations;
  h->nsub = subbands;
  h->npol = pols;
  h->G = subbands * pols;
  h->nchan = nchan;
  h->N = 2 * nchan;
  h->tint = tint_s;
  h->spi = llround(h->fs * tint_s);
  h->nu0.assign(subbands, 0.0);
  h->st.resize(stations);
  cudaError_t e = cudaGetDevice(&h->dev);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->own_stream, cudaStreamNonBlocking);
  for (int q = 0; q < kCopyStreams && e == cudaSuccess; ++q)
    e = cudaStreamCreateWithFlags(&h->copy_stream[q], cudaStreamNonBlocking);
  // the X step's stream gets the highest priority: its CTAs are placed first
  // as the F step's retire, so the two overlap instead of running in turn
  int prio_lo = 0, prio_hi = 0;
  if (e == cudaSuccess) e = cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
  if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&h->xstream, cudaStreamNonBlocking, prio_hi);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->dstream, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    g_create_error = std::string("corr_create: ") + cudaGetErrorString(e);
    cudaGetLastError();
    if (h->own_stream) cudaStreamDestroy(h->own_stream);
    for (int q = 0; q < kCopyStreams; ++q)
      if (h->copy_stream[q]) cudaStreamDestroy(h->copy_stream[q]);
    if (h->xstream) cudaStreamDestroy(h->xstream);
    if (h->dstream) cudaStreamDestroy(h->dstream);
    delete h;
    return CORR_ECUDA;
  }
  h->stream = h->own_stream;
  *hp = h;
  return CORR_OK;
}

int corr_set_format(corr_t* h, double fs_hz, const float lut[4]) {
  if (!h) return CORR_EINVAL;
  if (h->prepared) return h->fail(CORR_ESTATE, "corr_set_format: only before the first correlate");
  if (!(fs_hz > 0.0) || !isfinite(fs_hz)) return h->fail(CORR_EINVAL, "corr_set_format: fs must be > 0");
  const double spi = fs_hz * h->tint;
  const int64_t ispi = llround(spi);
  if (fabs(spi - (double)ispi) > 1e-6 || ispi < h->N)
    return h->fail(CORR_EINVAL, "corr_set_format: fs*tint must be a whole number of samples >= 2*nchan");
  if (lut)
    for (int q = 0; q < 4; ++q)
      if (!isfinite(lut[q])) return h->fail(CORR_EINVAL, "corr_set_format: level table must be finite");
  h->fs = fs_hz;
  h->spi = ispi;
  if (lut) memcpy(h->lut, lut, sizeof(h->lut));
  return CORR_OK;
}

int corr_set_sky_freq(corr_t* h, int subband, double nu0_hz) {
  if (!h) return CORR_EINVAL;
  if (subband < 0 || subband >= h->nsub) return h->fail(CORR_EINVAL, "corr_set_sky_freq: subband out of range");
  if (!isfinite(nu0_hz)) return h->fail(CORR_EINVAL, "corr_set_sky_freq: frequency must be finite");
  h->nu0[subband] = nu0_hz;
  h->polys_dirty = true;
  return CORR_OK;
}

int corr_set_precision(corr_t* h, int mode) {
  if (!h) return CORR_EINVAL;
  if (mode != CORR_PREC_FP32 && mode != CORR_PREC_FP16_TC && mode != CORR_PREC_FP8_TC)
    return h->fail(CORR_EINVAL, "corr_set_precision: unknown mode %d", mode);
  if (mode != CORR_PREC_FP32 && x_stations(h) > 64)
    return h->fail(CORR_EINVAL, cross_of(h) ? "corr_set_precision: with both hands the tensor-core X step takes at most 32 stations"
                                            : "corr_set_precision: the tensor-core X step takes at most 64 stations");
  if (h->prepared && mode != h->precision)
    return h->fail(CORR_ESTATE, "corr_set_precision: only before the first correlate");
  h->precision = mode;
  return CORR_OK;
}

int corr_set_frame_format(corr_t* h, int payload_bytes) {
  if (!h) return CORR_EINVAL;
  if (payload_bytes < 0 || payload_bytes % 16)
    return h->fail(CORR_EINVAL, "corr_set_frame_format: payload bytes must be 0 or a positive multiple of 16");
  for (const Station& x : h->st)
    if (x.started) return h->fail(CORR_ESTATE, "corr_set_frame_format: only before any samples are pushed or attached");
  h->payload = payload_bytes;
  return CORR_OK;
}

int corr_set_pol_products(corr_t* h, int mode) {
  if (!h) return CORR_EINVAL;
  if (mode != CORR_POL_PARALLEL && mode != CORR_POL_CROSS)
    return h->fail(CORR_EINVAL, "corr_set_pol_products: unknown mode %d", mode);
  if (mode == CORR_POL_CROSS && h->npol != 2)
    return h->fail(CORR_EINVAL, "corr_set_pol_products: both hands need two polarisations");
  if (mode == CORR_POL_CROSS && h->precision != CORR_PREC_FP32 && 2 * h->S > 64)
    return h->fail(CORR_EINVAL, "corr_set_pol_products: with both hands the tensor-core X step takes at most 32 stations");
  if (h->prepared && mode != h->pol_products)
    return h->fail(CORR_ESTATE, "corr_set_pol_products: only before the first correlate");
  h->pol_products = mode;
  return CORR_OK;
}

int corr_set_fringe_rotation(corr_t* h, int mode) {
  if (!h) return CORR_EINVAL;
  if (mode != CORR_ROT_POST_F && mode != CORR_ROT_PRE_F)
    return h->fail(CORR_EINVAL, "corr_set_fringe_rotation: unknown mode %d", mode);
  if (mode == CORR_ROT_PRE_F && !fstage_pre_supported(h->nchan))
    return h->fail(CORR_EINVAL, "corr_set_fringe_rotation: pre-F rotation takes at most 4096 channels");
  if (h->prepared && mode != h->rotation)
    return h->fail(CORR_ESTATE, "corr_set_fringe_rotation: only before the first correlate");
  h->rotation = mode;
  return CORR_OK;
}

int corr_set_x_unit(corr_t* h, int unit) {
  if (!h) return CORR_EINVAL;
  if (unit != CORR_X_AUTO && unit != CORR_X_CUDA_CORES && unit != CORR_X_TENSOR_CORES)
    return h->fail(CORR_EINVAL, "corr_set_x_unit: unknown unit %d", unit);
  if (h->prepared && unit != h->x_unit) return h->fail(CORR_ESTATE, "corr_set_x_unit: only before the first correlate");
  h->x_unit = unit;
  return CORR_OK;
}

int corr_set_pipeline(corr_t* h, int overlap) {
  if (!h) return CORR_EINVAL;
  if (overlap != 0 && overlap != 1) return h->fail(CORR_EINVAL, "corr_set_pipeline: overlap must be 0 or 1");
  if (h->prepared && overlap != h->pipeline)
    return h->fail(CORR_ESTATE, "corr_set_pipeline: only before the first correlate");
  h->pipeline = overlap;
  return CORR_OK;
}

int corr_set_chunk_blocks(corr_t* h, int blocks) {
  if (!h) return CORR_EINVAL;
  if (h->prepared) return h->fail(CORR_ESTATE, "corr_set_chunk_blocks: only before the first correlate");
  if (blocks < 0) return h->fail(CORR_EINVAL, "corr_set_chunk_blocks: blocks must be >= 0");
  h->chunk_req = blocks;
  return CORR_OK;
}

int corr_set_stream(corr_t* h, void* s) {
  if (!h) return CORR_EINVAL;
  h->stream = s ? (cudaStream_t)s : h->own_stream;
  return CORR_OK;
}

int corr_set_delay_poly(corr_t* h, int station, double t0_s, const double coeffs[6]) {
  if (!h) return CORR_EINVAL;
  if (station < 0 || station >= h->S) return h->fail(CORR_EINVAL, "corr_set_delay_poly: station out of range");
  if (!coeffs || !isfinite(t0_s)) return h->fail(CORR_EINVAL, "corr_set_delay_poly: bad t0 or coeffs");
  for (int q = 0; q < 6; ++q)
    if (!isfinite(coeffs[q])) return h->fail(CORR_EINVAL, "corr_set_delay_poly: coefficients must be finite");
  Station& s = h->st[station];
  if (!s.segs.empty() && !(t0_s > s.segs.back().t0))
    return h->fail(CORR_EINVAL, "corr_set_delay_poly: t0 must increase (station %d)", station);
  if ((int)s.segs.size() >= kMaxSegs) return h->fail(CORR_EINVAL, "corr_set_delay_poly: at most 64 segments");
  Seg g;
  g.t0 = t0_s;
  memcpy(g.c, coeffs, sizeof(g.c));
  s.segs.push_back(g);
  h->polys_dirty = true;
  return CORR_OK;
}

int corr_set_stream_start(corr_t* h, int station, int64_t first_sample) {
  if (!h) return CORR_EINVAL;
  if (station < 0 || station >= h->S) return h->fail(CORR_EINVAL, "corr_set_stream_start: station out of range");
  if (h->st[station].started) return h->fail(CORR_ESTATE, "corr_set_stream_start: station already has data");
  h->st[station].sample0 = first_sample;
  return CORR_OK;
}

static int grow(corr_t* h, Station& s, size_t need) {
  if (need <= s.cap) return CORR_OK;
  size_t cap = s.cap ? s.cap : ((size_t)1 << 20);
  while (cap < need) cap *= 2;
  uint8_t* nb = nullptr;
  int rc = dalloc(h, (void**)&nb, cap, "station stream");
  if (rc) return rc;
  if (s.len) {
    cudaError_t e = cudaMemcpyAsync(nb, s.dbuf, s.len, cudaMemcpyDeviceToDevice, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
      cudaFree(nb);
      return h->cuda_fail(e, "stream grow copy");
    }
  }
  cudaFree(s.dbuf);
  s.dbuf = nb;
  s.cap = cap;
  return CORR_OK;
}

int corr_reserve(corr_t* h, int station, size_t nbytes) {
  if (!h) return CORR_EINVAL;
  if (station < 0 || station >= h->S) return h->fail(CORR_EINVAL, "corr_reserve: station out of range");
  if (h->st[station].attached) return h->fail(CORR_ESTATE, "corr_reserve: station uses attached memory");
  int rc = use_device(h);
  if (rc) return rc;
  return grow(h, h->st[station], nbytes);
}

int corr_push_samples(corr_t* h, int station, const void* bytes, size_t nbytes) {
  if (!h) return CORR_EINVAL;
  if (station < 0 || station >= h->S) return h->fail(CORR_EINVAL, "corr_push_samples: station out of range");
  if (nbytes % 4) return h->fail(CORR_EINVAL, "corr_push_samples: nbytes must be a multiple of 4");
  if (nbytes && !bytes) return h->fail(CORR_EINVAL, "corr_push_samples: bytes is NULL");
  Station& s = h->st[station];
  if (s.attached) return h->fail(CORR_ESTATE, "corr_push_samples: station uses attached device memory");
  if (h->flushed) return h->fail(CORR_ESTATE, "corr_push_samples: after corr_flush");
  int rc = use_device(h);
  if (rc) return rc;
  if (!s.pending.empty() && (rc = drain_pushes(h))) return rc;
  if ((rc = grow(h, s, s.len + nbytes))) return rc;
  if (nbytes) {
    CK(cudaMemcpyAsync(s.dbuf + s.len, bytes, nbytes, cudaMemcpyHostToDevice, h->stream), "push H2D");
    CK(cudaStreamSynchronize(h->stream), "push sync");
  }
  s.len += nbytes;
  s.started = true;
  return CORR_OK;
}

int corr_push_samples_async(corr_t* h, int station, const void* bytes, size_t nbytes) {
  if (!h) return CORR_EINVAL;
  if (station < 0 || station >= h->S) return h->fail(CORR_EINVAL, "corr_push_samples_async: station out of range");
  if (nbytes % 4) return h->fail(CORR_EINVAL, "corr_push_samples_async: nbytes must be a multiple of 4");
  if (nbytes && !bytes) return h->fail(CORR_EINVAL, "corr_push_samples_async: bytes is NULL");
  Station& s = h->st[station];
  if (s.attached) return h->fail(CORR_ESTATE, "corr_push_samples_async: station uses attached device memory");
  if (h->flushed) return h->fail(CORR_ESTATE, "corr_push_samples_async: after corr_flush");
  int rc = use_device(h);
  if (rc) return rc;
  if (s.len + nbytes > s.cap) {
    // growing moves the buffer: let every copy into it finish first
    if ((rc = drain_pushes(h))) return rc;
    CK(cudaStreamSynchronize(h->stream), "sync before stream growth");
    if ((rc = grow(h, s, s.len + nbytes))) return rc;
  }
  for (size_t o = 0; o < nbytes; o += kCopyPiece) {
    const size_t n = nbytes - o < kCopyPiece ? nbytes - o : kCopyPiece;
    cudaStream_t cs = h->copy_stream[h->copy_next];
    h->copy_next = (h->copy_next + 1) % kCopyStreams;
    cudaEvent_t ev = nullptr;
    CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), "push event");
    cudaError_t e = cudaMemcpyAsync(s.dbuf + s.len + o, (const uint8_t*)bytes + o, n, cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess) e = cudaEventRecord(ev, cs);
    if (e != cudaSuccess) {
      cudaEventDestroy(ev);
      return h->cuda_fail(e, "asynchronous push");
    }
    s.pending.push_back({s.len + o, s.len + o + n, ev});
  }
  s.len += nbytes;
  s.started = true;
  return CORR_OK;
}

int corr_wait_pushes(corr_t* h) {
  if (!h) return CORR_EINVAL;
  int rc = use_device(h);
  if (rc) return rc;
  return drain_pushes(h);
}

int corr_attach_samples_device(corr_t* h, int station, const void* dev_bytes, size_t nbytes) {
  if (!h) return CORR_EINVAL;
  if (station < 0 || station >= h->S) return h->fail(CORR_EINVAL, "corr_attach_samples_device: station out of range");
  if (nbytes % 4) return h->fail(CORR_EINVAL, "corr_attach_samples_device: nbytes must be a multiple of 4");
  if (!dev_bytes || ((uintptr_t)dev_bytes & 15))
    return h->fail(CORR_EINVAL, "corr_attach_samples_device: pointer must be non-NULL and 16-byte aligned");
  Station& s = h->st[station];
  if (s.started) return h->fail(CORR_ESTATE, "corr_attach_samples_device: station already has data");
  int rc = use_device(h);
  if (rc) return rc;
  cudaPointerAttributes at;
  cudaError_t e = cudaPointerGetAttributes(&at, dev_bytes);
  if (e != cudaSuccess || at.type != cudaMemoryTypeDevice || at.device != h->dev) {
    cudaGetLastError();
    return h->fail(CORR_EINVAL, "corr_attach_samples_device: not device memory of the handle's device");
  }
  cudaFree(s.dbuf);
  s.dbuf = nullptr;
  s.cap = 0;
  s.ext = (const uint8_t*)dev_bytes;
  s.len = nbytes;
  s.attached = true;
  s.started = true;
  return CORR_OK;
}

int corr_attach_samples_host(corr_t* h, int station, const void* host_bytes, size_t nbytes) {
  if (!h) return CORR_EINVAL;
  if (station < 0 || station >= h->S) return h->fail(CORR_EINVAL, "corr_attach_samples_host: station out of range");
  if (nbytes % 4) return h->fail(CORR_EINVAL, "corr_attach_samples_host: nbytes must be a multiple of 4");
  if (!host_bytes || ((uintptr_t)host_bytes & 15))
    return h->fail(CORR_EINVAL, "corr_attach_samples_host: pointer must be non-NULL and 16-byte aligned");
  Station& s = h->st[station];
  if (s.started) return h->fail(CORR_ESTATE, "corr_attach_samples_host: station already has data");
  int rc = use_device(h);
  if (rc) return rc;
  cudaPointerAttributes at;
  cudaError_t e = cudaPointerGetAttributes(&at, host_bytes);
  if (e != cudaSuccess || at.type != cudaMemoryTypeHost || !at.devicePointer) {
    cudaGetLastError();
    return h->fail(CORR_EINVAL, "corr_attach_samples_host: not pinned (page-locked, mapped) host memory");
  }
  cudaFree(s.dbuf);
  s.dbuf = nullptr;
  s.cap = 0;
  s.ext = (const uint8_t*)at.devicePointer;  // the device-side address of the pinned pages
  s.host = true;
  s.len = nbytes;
  s.attached = true;
  s.started = true;
  return CORR_OK;
}

int corr_flush(corr_t* h) {
  if (!h) return CORR_EINVAL;
  h->flushed = true;
  return CORR_OK;
}

int corr_correlate(corr_t* h, float* out, double* weights) {
  if (!h) return CORR_EINVAL;
  if (!out) return h->fail(CORR_EINVAL, "corr_correlate: out is NULL");
  int rc = use_device(h);
  if (rc) return rc;
  if ((rc = prepare(h))) return rc;
  double* dw = weights ? h->d_wts : nullptr;
  rc = run_integration(h, h->d_out, dw);
  if (rc == CORR_OK) {
    const size_t bytes = sizeof(float2) * (size_t)nbl_of(h->S) * out_per_baseline(h);
    cudaError_t e = cudaMemcpyAsync(out, h->d_out, bytes, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess && dw)
      e = cudaMemcpyAsync(weights, dw, sizeof(double) * nbl_of(h->S), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) rc = h->cuda_fail(e, "correlate D2H");
    else if (*h->h_err) rc = h->fail(CORR_ETIMEOUT, "an X-step wait timed out on the device");
  }
  return rc;
}

int corr_correlate_device(corr_t* h, float* dev_out, double* dev_weights) {
  if (!h) return CORR_EINVAL;
  if (!dev_out) return h->fail(CORR_EINVAL, "corr_correlate_device: dev_out is NULL");
  return run_integration(h, reinterpret_cast<float2*>(dev_out), dev_weights);
}

int corr_next_integration(const corr_t* h, int64_t* index) {
  if (!h || !index) return CORR_EINVAL;
  *index = h->next_int;
  return CORR_OK;
}

int corr_rewind(corr_t* h) {
  if (!h) return CORR_EINVAL;
  h->next_int = 0;
  return CORR_OK;  // a look-ahead for another integration is dropped by the next correlate
}

int corr_reset(corr_t* h) {
  if (!h) return CORR_EINVAL;
  int rc = use_device(h);
  if (rc) return rc;
  cudaStreamSynchronize(h->stream);
  if (h->xstream) cudaStreamSynchronize(h->xstream);
  drop_lookahead(h);
  drain_pushes(h);
  for (Station& s : h->st) {
    for (auto& pe : s.pending) cudaEventDestroy(pe.ev);
    s.pending.clear();
    if (s.attached) {
      s.ext = nullptr;
      s.attached = false;
      s.host = false;
      s.len = 0;
    } else {
      s.len = 0;
    }
    s.nframes_done = 0;
    s.started = false;
  }
  h->flushed = false;
  h->next_int = 0;
  // a device wait that timed out earlier no longer blocks the handle
  if (h->prepared) {
    cudaError_t e = cudaMemsetAsync(h->d_err, 0, sizeof(int), h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return h->cuda_fail(e, "corr_reset: error flag");
    *h->h_err = 0;
  }
  return CORR_OK;
}

const char* corr_last_error(const corr_t* h) {
  if (!h) return g_create_error.c_str();
  return h->err.c_str();
}

void corr_destroy(corr_t* h) {
  if (!h) return;
  int cur = -1;
  cudaGetDevice(&cur);
  if (cur != h->dev) cudaSetDevice(h->dev);
  if (h->stream) cudaStreamSynchronize(h->stream);
  if (h->xstream) cudaStreamSynchronize(h->xstream);
  if (h->dstream) cudaStreamSynchronize(h->dstream);
  drain_pushes(h);
  for (Station& s : h->st) {
    for (auto& pe : s.pending) cudaEventDestroy(pe.ev);
    cudaFree(s.dbuf);
    cudaFree(s.pay);
    cudaFree(s.fok);
  }
  for (auto& m : h->marks) {
    cudaEventDestroy(m.a);
    cudaEventDestroy(m.b);
  }
  for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
  free_device(h);
  if (h->own_stream) cudaStreamDestroy(h->own_stream);
  if (h->xstream) cudaStreamDestroy(h->xstream);
  if (h->dstream) cudaStreamDestroy(h->dstream);
  for (int q = 0; q < kCopyStreams; ++q)
    if (h->copy_stream[q]) cudaStreamDestroy(h->copy_stream[q]);
  if (cur != h->dev && cur >= 0) cudaSetDevice(cur);
  delete h;
}

// ---- several handles in one CUDA graph -----------------------------------------

namespace {
constexpr int kBatchStreams = 16;
// per-device streams, events and the last instantiated graph of corr_batch_run
struct BatchCtx {
  bool ready = false;
  cudaStream_t st[kBatchStreams] = {};
  cudaEvent_t fork = nullptr, done = nullptr, join[kBatchStreams] = {};
  cudaGraphExec_t exec = nullptr;
};
BatchCtx g_batch[64];
std::mutex g_batch_mu;
}  // namespace

int corr_batch_run(corr_t* const* hs, int n, float* const* dev_out, double* const* dev_weights, void* cuda_stream) {
  if (!hs || n < 1 || !dev_out) return CORR_EINVAL;
  for (int j = 0; j < n; ++j)
    if (!hs[j] || !dev_out[j]) return CORR_EINVAL;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return CORR_ECUDA;
  for (int j = 0; j < n; ++j) {
    corr_t* h = hs[j];
    for (int k = 0; k < j; ++k)
      if (hs[k] == h) return h->fail(CORR_EINVAL, "corr_batch_run: a handle appears twice");
    if (h->dev != dev) return h->fail(CORR_EINVAL, "corr_batch_run: handles must live on the current device");
    if (!h->flushed) return h->fail(CORR_ESTATE, "corr_batch_run: call corr_flush on every handle first");
    if (h->profiling) return h->fail(CORR_ESTATE, "corr_batch_run: profiling must be off");
  }
  std::lock_guard<std::mutex> lk(g_batch_mu);
  BatchCtx& b = g_batch[dev];
  cudaError_t e = cudaSuccess;
  if (!b.ready) {
    for (int q = 0; q < kBatchStreams && e == cudaSuccess; ++q)
      e = cudaStreamCreateWithFlags(&b.st[q], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b.fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b.done, cudaEventDisableTiming);
    for (int q = 0; q < kBatchStreams && e == cudaSuccess; ++q)
      e = cudaEventCreateWithFlags(&b.join[q], cudaEventDisableTiming);
    if (e != cudaSuccess) return hs[0]->cuda_fail(e, "corr_batch_run: streams");
    b.ready = true;
  }
  // everything that waits on the host or allocates happens before the capture
  for (int j = 0; j < n; ++j) {
    corr_t* h = hs[j];
    int rc;
    if ((rc = prepare(h)) || (rc = upload_model(h)) || (rc = drain_pushes(h)) || (rc = drop_lookahead(h))) return rc;
    for (Station& x : h->st) {
      for (auto& pe : x.pending) cudaEventDestroy(pe.ev);
      x.pending.clear();
    }
    CK(cudaStreamSynchronize(h->stream), "corr_batch_run: handle stream");
    CK(cudaStreamSynchronize(h->xstream), "corr_batch_run: handle stream");
    if (*h->h_err) return h->fail(CORR_ETIMEOUT, "an X-step wait timed out on the device");
  }
  cudaStream_t root = cuda_stream ? (cudaStream_t)cuda_stream : b.st[0];
  cudaGraph_t graph = nullptr;
  e = cudaStreamBeginCapture(root, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return hs[0]->cuda_fail(e, "corr_batch_run: begin capture");
  int rc = CORR_OK, bad = 0;
  // fork: every branch stream joins the capture behind the root
  e = cudaEventRecord(b.fork, root);
  for (int q = 0; q < kBatchStreams && e == cudaSuccess; ++q)
    if (b.st[q] != root) e = cudaStreamWaitEvent(b.st[q], b.fork, 0);
  for (int j = 0; j < n && e == cudaSuccess && rc == CORR_OK; ++j) {
    corr_t* h = hs[j];
    cudaStream_t st = b.st[j % kBatchStreams];
    const int64_t i = h->next_int;
    const int64_t bfirst = integ_first_block(h, i);
    const int M = (int)(integ_first_block(h, i + 1) - bfirst);
    bad = j;
    const int slot = (int)(i & 1);
    e = launch_delay_blocks(delay_params(h, bfirst, M, h->Mcap, slot), st);
    if (e != cudaSuccess) break;
    // one stream per scan inside the graph (scans run side by side instead)
    rc = enqueue_rest(h, st, M, reinterpret_cast<float2*>(dev_out[j]), dev_weights ? dev_weights[j] : nullptr, slot,
                      false);
    if (rc == CORR_OK) e = cudaMemcpyAsync(h->h_err, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, st);
  }
  // join every branch back into the root
  for (int q = 0; q < kBatchStreams && e == cudaSuccess; ++q) {
    if (b.st[q] == root) continue;
    e = cudaEventRecord(b.join[q], b.st[q]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(root, b.join[q], 0);
  }
  cudaError_t e2 = cudaStreamEndCapture(root, &graph);
  if (e == cudaSuccess) e = e2;
  if (rc != CORR_OK || e != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    return rc != CORR_OK ? rc : hs[bad]->cuda_fail(e, "corr_batch_run: capture");
  }
  // reuse the executable graph when only parameters changed
  if (b.exec) {
    cudaGraphExecUpdateResultInfo info;
    if (cudaGraphExecUpdate(b.exec, graph, &info) != cudaSuccess) {
      cudaGetLastError();
      cudaGraphExecDestroy(b.exec);
      b.exec = nullptr;
    }
  }
  if (!b.exec) e = cudaGraphInstantiate(&b.exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e == cudaSuccess) e = cudaGraphLaunch(b.exec, root);
  if (e == cudaSuccess) e = cudaEventRecord(b.done, root);
  // later work on each handle's own stream comes after the graph
  for (int j = 0; j < n && e == cudaSuccess; ++j) e = cudaStreamWaitEvent(hs[j]->stream, b.done, 0);
  if (e != cudaSuccess) {
    if (b.exec) cudaGraphExecDestroy(b.exec);
    b.exec = nullptr;
    return hs[0]->cuda_fail(e, "corr_batch_run: graph launch");
  }
  for (int j = 0; j < n; ++j) hs[j]->next_int += 1;
  return CORR_OK;
}

int corr_device_bytes(corr_t* h, size_t* bytes) {
  if (!h || !bytes) return CORR_EINVAL;
  WorkLayout w;
  int rc = work_layout(h, w);
  if (rc) return rc;
  size_t total = w.total();
  for (const Station& x : h->st) {
    if (!x.attached) total += x.cap;  // sample buffers the handle owns
    if (h->payload > 0)               // deframed payloads and their flags
      total += std::max(x.pay_cap, (size_t)station_frames(h, x) * h->payload) +
               std::max(x.fok_cap, (size_t)station_frames(h, x));
  }
  *bytes = total;
  return CORR_OK;
}

// ---- inspection ------------------------------------------------------------

int corr_set_profiling(corr_t* h, int enable) {
  if (!h) return CORR_EINVAL;
  h->profiling = enable != 0;
  return CORR_OK;
}

int corr_read_profile(corr_t* h, double ms[4], int64_t launches[4]) {
  if (!h || !ms || !launches) return CORR_EINVAL;
  int rc = use_device(h);
  if (rc || (rc = prof_collect(h))) return rc;
  for (int q = 0; q < kStages; ++q) {
    ms[q] = h->prof_ms[q];
    launches[q] = h->prof_n[q];
    h->prof_ms[q] = 0.0;
    h->prof_n[q] = 0;
  }
  return CORR_OK;
}

int corr_launch_shape(const corr_t* h, int* chunk_blocks, int* kz) {
  if (!h || !chunk_blocks || !kz) return CORR_EINVAL;
  *chunk_blocks = h->CB;
  *kz = h->KZ;
  return CORR_OK;
}

int corr_debug_set_wait_limit(long long spins) {
  set_wait_limit(spins);
  return CORR_OK;
}

int corr_debug_delays(corr_t* h, int64_t b0, int64_t nb, int64_t* start, double* eps, double* tau,
                      uint8_t* valid) {
  if (!h) return CORR_EINVAL;
  if (nb <= 0 || nb > (1 << 24)) return h->fail(CORR_EINVAL, "corr_debug_delays: nb must be 1..2^24");
  int rc;
  if ((rc = use_device(h)) || (rc = prepare(h)) || (rc = upload_model(h))) return rc;
  const int S = h->S;
  int64_t* d_start = nullptr;
  float* d_delta = nullptr;
  float* d_phi = nullptr;
  float2* d_dphi = nullptr;  // pre-F: phase step per sample (hi, lo), [S][nsub][Mcap]
  uint8_t* d_valid = nullptr;
  double *d_eps = nullptr, *d_tau = nullptr;
  const size_t n = (size_t)S * nb;
  if ((rc = dalloc(h, (void**)&d_start, n * 8, "dbg")) || (rc = dalloc(h, (void**)&d_delta, n * 4, "dbg")) ||
      (rc = dalloc(h, (void**)&d_phi, n * 4 * h->nsub, "dbg")) || (rc = dalloc(h, (void**)&d_valid, n, "dbg")) ||
      (rc = dalloc(h, (void**)&d_eps, n * 8, "dbg")) || (rc = dalloc(h, (void**)&d_tau, n * 8, "dbg"))) {
    cudaFree(d_start); cudaFree(d_delta); cudaFree(d_phi); cudaFree(d_valid); cudaFree(d_eps); cudaFree(d_tau);
    return rc;
  }
  DelayParams p = delay_params(h, b0, (int)nb, (int)nb, 0);
  p.start = d_start;
  p.delta = d_delta;
  p.phi = d_phi;
  p.valid = d_valid;
  p.eps_out = d_eps;
  p.tau_out = d_tau;
  p.dphi = nullptr;  // phi: the phase at the block centre
  cudaError_t e = launch_delay_blocks(p, h->stream);
  if (e == cudaSuccess && start) e = cudaMemcpyAsync(start, d_start, n * 8, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess && eps) e = cudaMemcpyAsync(eps, d_eps, n * 8, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess && tau) e = cudaMemcpyAsync(tau, d_tau, n * 8, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess && valid) e = cudaMemcpyAsync(valid, d_valid, n, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  cudaFree(d_start); cudaFree(d_delta); cudaFree(d_phi); cudaFree(d_valid); cudaFree(d_eps); cudaFree(d_tau);
  if (e != cudaSuccess) return h->cuda_fail(e, "corr_debug_delays");
  return CORR_OK;
}

int corr_debug_codes(corr_t* h, int station, int stream, int64_t t0, int64_t count, uint8_t* codes) {
  if (!h) return CORR_EINVAL;
  if (station < 0 || station >= h->S || stream < 0 || stream >= h->G || count < 0 || !codes)
    return h->fail(CORR_EINVAL, "corr_debug_codes: bad argument");
  int rc;
  if ((rc = use_device(h)) || (rc = prepare(h)) || (rc = upload_model(h))) return rc;
  uint8_t* d = nullptr;
  if ((rc = dalloc(h, (void**)&d, (size_t)count, "dbg codes"))) return rc;
  cudaError_t e = launch_unpack_codes(h->d_views, station, h->G, stream, t0, count, d, h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(codes, d, (size_t)count, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  cudaFree(d);
  if (e != cudaSuccess) return h->cuda_fail(e, "corr_debug_codes");
  return CORR_OK;
}

int corr_debug_spectrum(corr_t* h, int station, int stream, int64_t block, float* out, int* valid) {
  if (!h) return CORR_EINVAL;
  if (station < 0 || station >= h->S || stream < 0 || stream >= h->G || !out)
    return h->fail(CORR_EINVAL, "corr_debug_spectrum: bad argument");
  int rc;
  if ((rc = use_device(h)) || (rc = prepare(h)) || (rc = upload_model(h)) || (rc = drop_lookahead(h))) return rc;
  // one-block pass through the same kernels, in the handle's work buffers
  // (descriptor slot 0, which the next correlate call fills again)
  DelayParams dp = delay_params(h, block, 1, h->Mcap, 0);
  CK(launch_delay_blocks(dp, h->stream), "delay_blocks");
  // a buffer of its own: in tensor-core tile mode the handle has no FP32
  // spectra buffer
  float2* spec = nullptr;
  if ((rc = dalloc(h, (void**)&spec, sizeof(float2) * (size_t)h->G * h->S * h->nchan, "debug spectrum"))) return rc;
  FParams fp = fparams(h, 0, 1, 0);
  fp.out = spec;
  fp.cross = 0;  // [stream][block][station]
  cudaError_t e = launch_fstage(fp, h->stream);
  const float2* src = spec + ((size_t)stream * 1 * h->S + station) * h->nchan;
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(out, src, sizeof(float2) * h->nchan, cudaMemcpyDeviceToHost, h->stream);
  uint8_t v = 0;
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&v, h->d_valid[0] + (size_t)station * h->Mcap, 1, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  cudaFree(spec);
  if (e != cudaSuccess) return h->cuda_fail(e, "corr_debug_spectrum");
  if (valid) *valid = v;
  return CORR_OK;
}

}  // extern "C"
