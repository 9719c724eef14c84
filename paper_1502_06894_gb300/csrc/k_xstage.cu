// k_xstage.cu -- the X step of the FX correlator on CUDA cores in FP32 (the
// paper, Abstract: after the Fourier transform every station pair is
// cross-multiplied).  For each stream g and channel k, over the FFT blocks of
// a chunk:  V_ab[k] += X_a[k] conj(X_b[k]) for every baseline a <= b
// (autocorrelations included, parallel hands only).
//
// One thread owns one channel of one stream and a TA x TA tile of baselines
// (a diagonal tile keeps only a <= b), so each loaded spectrum value is used
// TA times from registers.  The blocks of a chunk are split into KZ ranges;
// each range sums at most 256 blocks in registers and then adds that partial
// into its own FP32 accumulator slice part[kz], in a fixed order, so results
// are deterministic and the FP32 sums stay short (hierarchical accumulation).
#include "corr_internal.cuh"

#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <type_traits>
#include <cudaTypedefs.h>

namespace corr {

constexpr int kXT = 128;  // threads per CTA (channels)

// 16-byte asynchronous copy to shared memory; src_bytes = 0 writes zeros.
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, int src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes));
}

// acc + x conj(y) on packed FP32 pairs: acc + x (y.x, y.x) + xr (y.y, y.y)
// with xr = (x.y, -x.x), formed once per loaded value: two f32x2 fused
// multiply-adds per baseline instead of four scalar ones.
__device__ __forceinline__ float2 cmac_conj(float2 acc, float2 x, float2 xr, float2 y) {
  return __ffma2_rn(xr, make_float2(y.y, y.y), __ffma2_rn(x, make_float2(y.x, y.x), acc));
}
__device__ __forceinline__ float2 rot_conj(float2 x) { return __fmul2_rn(make_float2(x.y, x.x), make_float2(1.f, -1.f)); }
// An autocorrelation needs only |x|^2: the accumulator keeps (sum re^2,
// sum im^2), one f32x2 FMA per block; auto_value() forms the visibility.
__device__ __forceinline__ float2 cmac_auto(float2 acc, float2 x) { return __ffma2_rn(x, x, acc); }
__device__ __forceinline__ float2 auto_value(float2 acc) { return make_float2(acc.x + acc.y, 0.f); }

// The tile pairs of one 128-channel tile are consecutive CTAs (blockIdx.x
// = channel tile x pairs + pair), so the pairs that read the same stations'
// spectra run side by side and all but the first read come from L2.  The
// diagonal pairs (DIAG) and the off-diagonal ones are separate launches.
// The 2 x 8 stations' values of each block reach shared memory through a
// cp.async ring of kStagesT blocks, so that many blocks' loads are in flight
// without registers (the accumulators take 128 of them).
// First tile row of part `part` of `npart` for a triangular tile: the parts
// get about equal numbers of baselines (row i holds TA - i of them).
__host__ __device__ constexpr int tri_split(int TA, int npart, int part) {
  if (part <= 0) return 0;
  if (part >= npart) return TA;
  int acc = 0, i = 0;
  const int total = TA * (TA + 1) / 2;
  while (i < TA && 2 * npart * (acc + (TA - i)) <= 2 * total * part + npart * (TA - i)) {
    acc += TA - i;
    ++i;
  }
  return i;
}

constexpr int kStagesT = 4;

// Two threads per channel: thread part 0 takes tile rows [0, SPLIT) and
// part 1 rows [SPLIT, TA) (half the baselines each), so a thread holds 32
// accumulators instead of 64 and an SM runs twice the warps.
template <int TA, bool DIAG>
__global__ void __launch_bounds__(2 * kXT) k_xmac(XParams p, int ntile) {
  extern __shared__ __align__(16) unsigned char xt_raw[];
  constexpr int NT = DIAG ? 1 : 2;                 // station tiles per block
  float2* ring = reinterpret_cast<float2*>(xt_raw);  // [kStagesT][NT][TA][kXT]
  const int npo = DIAG ? ntile : ntile * (ntile - 1) / 2;  // pairs of this launch
  const int pidx = blockIdx.x % npo;
  const int k0 = (blockIdx.x / npo) * kXT;
  const int lane = threadIdx.x % kXT;
  const int part = threadIdx.x / kXT;
  const int k = k0 + lane;
  const int g = blockIdx.y;
  const int kz = blockIdx.z;
  int ta = pidx, tb = pidx;
  if (!DIAG) {  // off-diagonal pair pidx in row-major order over ta < tb
    int q = pidx;
    ta = 0;
    while (q >= ntile - 1 - ta) { q -= ntile - 1 - ta; ++ta; }
    tb = ta + 1 + q;
  }
  const int S = p.S;
  const int b_lo = (int)((int64_t)p.CB * kz / p.KZ);
  const int b_hi = (int)((int64_t)p.CB * (kz + 1) / p.KZ);
  if (b_hi <= b_lo) return;
  const int nb = b_hi - b_lo;
  constexpr int stage_elems = NT * TA * kXT;
  const uint32_t ring_s = (uint32_t)__cvta_generic_to_shared(ring);
  const size_t sstride = (size_t)p.nchan;

  // copies of block b_lo + q into slot q % kStagesT: NT x TA rows of 128
  // channels, 64 pieces of 16 bytes each; rows beyond S and channels beyond
  // nchan are zero-filled
  auto issue = [&](int q) {
    if (q < nb) {
      const int slot = q % kStagesT;
      const int b = b_lo + q;
      for (int e = threadIdx.x; e < NT * TA * 64; e += 2 * kXT) {
        const int piece = e & 63;
        const int row = e >> 6;                     // (tile, station in tile)
        const int st = ((row >= TA) ? tb : ta) * TA + (row % TA);
        const int ch = k0 + piece * 2;
        const bool in = st < S && ch < p.nchan;
        const float2* src = p.spec + ((size_t)g * p.CB + b) * (size_t)S * sstride + (size_t)(in ? st : 0) * sstride +
                            (in ? ch : 0);
        const uint32_t dst = ring_s + (uint32_t)((slot * stage_elems + row * kXT + piece * 2) * 8);
        cp_async16(dst, src, in ? 16 : 0);
      }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };

  auto run = [&](auto I0c, auto I1c) {
    constexpr int I0 = decltype(I0c)::value, I1 = decltype(I1c)::value;
    float2 acc[TA][TA];
#pragma unroll
    for (int i = I0; i < I1; ++i)
#pragma unroll
      for (int j = 0; j < TA; ++j) acc[i][j] = make_float2(0.f, 0.f);

    for (int q = 0; q < kStagesT - 1; ++q) issue(q);
    for (int q = 0; q < nb; ++q) {
      issue(q + kStagesT - 1);
      asm volatile("cp.async.wait_group %0;" ::"n"(kStagesT - 1) : "memory");
      __syncthreads();
      const float2* st = ring + (q % kStagesT) * stage_elems + lane;
      float2 a[TA], b[TA];
#pragma unroll
      for (int i = I0; i < (DIAG ? TA : I1); ++i) a[i] = st[i * kXT];
      if (!DIAG) {
#pragma unroll
        for (int i = 0; i < TA; ++i) b[i] = st[(TA + i) * kXT];
      }
#pragma unroll
      for (int i = I0; i < I1; ++i) {
        const float2 ar = rot_conj(a[i]);
#pragma unroll
        for (int j = DIAG ? i : 0; j < TA; ++j)
          acc[i][j] = (DIAG && j == i) ? cmac_auto(acc[i][j], a[i])
                                       : cmac_conj(acc[i][j], a[i], ar, DIAG ? a[j] : b[j]);  // X_a conj(X_b)
      }
      __syncthreads();
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    if (k >= p.nchan) return;
    const int nbl = nbl_of(S);
#pragma unroll
    for (int i = I0; i < I1; ++i)
#pragma unroll
      for (int j = DIAG ? i : 0; j < TA; ++j) {
        const int sa = ta * TA + i, sb = tb * TA + j;
        if (sa < S && sb < S) {
          float2* dst = p.part + (((size_t)kz * nbl + bl_index(sa, sb, S)) * p.G + g) * sstride + k;
          const float2 x = (DIAG && j == i) ? auto_value(acc[i][j]) : acc[i][j];
          float2 v = *dst;
          v.x += x.x;
          v.y += x.y;
          *dst = v;
        }
      }
  };
  constexpr int SPLIT = DIAG ? tri_split(TA, 2, 1) : TA / 2;
  if (part == 0)
    run(std::integral_constant<int, 0>{}, std::integral_constant<int, SPLIT>{});
  else
    run(std::integral_constant<int, SPLIT>{}, std::integral_constant<int, TA>{});
}

// For S <= 12 (one triangular tile of baselines per channel) the spectra
// reach the threads through a shared-memory ring filled by cp.async, so the
// number of bytes in flight no longer depends on how many registers the
// accumulators take: kStagesX stages of kNB blocks x S stations x 128
// channels, one CTA per (128-channel tile, stream, block range).
constexpr int kNB = 2;       // blocks per stage
constexpr int kStagesX = 4;  // ring depth


template <int TA>
__global__ void __launch_bounds__(kXT) k_xmac_ring(XParams p) {
  extern __shared__ __align__(16) unsigned char xs_raw[];
  float2* ring = reinterpret_cast<float2*>(xs_raw);  // [kStagesX][kNB][S][kXT]
  const int tid = threadIdx.x;
  const int k0 = blockIdx.x * kXT;
  const int k = k0 + tid;
  const int g = blockIdx.y;
  const int kz = blockIdx.z;
  const int S = p.S;
  const int b_lo = (int)((int64_t)p.CB * kz / p.KZ);
  const int b_hi = (int)((int64_t)p.CB * (kz + 1) / p.KZ);
  if (b_hi <= b_lo) return;
  const int nst = (b_hi - b_lo + kNB - 1) / kNB;  // stages of this CTA
  const int stage_elems = kNB * S * kXT;
  const uint32_t ring_s = (uint32_t)__cvta_generic_to_shared(ring);

  // issue the copies of stage q (blocks b_lo + q*kNB ...) into ring slot q % kStagesX
  auto issue = [&](int q) {
    if (q < nst) {
      const int slot = q % kStagesX;
      const int chunks = kNB * S * (kXT * 8 / 16);  // 16-byte pieces
      for (int c = tid; c < chunks; c += kXT) {
        const int row = c >> 6;                    // (block-in-stage, station), 64 pieces per row
        const int piece = c & 63;
        const int bi = row / S;
        const int st = row - bi * S;
        const int b = b_lo + q * kNB + bi;
        const int ch = k0 + piece * 2;
        const bool in = b < b_hi && ch < p.nchan;
        const float2* src = p.spec + ((size_t)g * p.CB + (in ? b : b_lo)) * (size_t)S * p.nchan +
                            (size_t)st * p.nchan + (in ? ch : 0);
        const uint32_t dst = ring_s + (uint32_t)(((slot * kNB + bi) * S + st) * kXT + piece * 2) * 8u;
        cp_async16(dst, src, in ? 16 : 0);
      }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };

  float2 acc[TA][TA];
#pragma unroll
  for (int i = 0; i < TA; ++i)
#pragma unroll
    for (int j = 0; j < TA; ++j) acc[i][j] = make_float2(0.f, 0.f);

#pragma unroll
  for (int q = 0; q < kStagesX - 1; ++q) issue(q);
  for (int q = 0; q < nst; ++q) {
    issue(q + kStagesX - 1);
    asm volatile("cp.async.wait_group %0;" ::"n"(kStagesX - 1) : "memory");
    __syncthreads();
    const float2* st = ring + (q % kStagesX) * stage_elems;
#pragma unroll
    for (int bi = 0; bi < kNB; ++bi) {
      float2 a[TA];
#pragma unroll
      for (int i = 0; i < TA; ++i) a[i] = i < S ? st[(bi * S + i) * kXT + tid] : make_float2(0.f, 0.f);
#pragma unroll
      for (int i = 0; i < TA; ++i) {
        const float2 ar = rot_conj(a[i]);
#pragma unroll
        for (int j = i; j < TA; ++j) acc[i][j] = j == i ? cmac_auto(acc[i][j], a[i]) : cmac_conj(acc[i][j], a[i], ar, a[j]);
      }
    }
    __syncthreads();
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
  if (k >= p.nchan) return;
  const int nbl = nbl_of(S);
#pragma unroll
  for (int i = 0; i < TA; ++i)
#pragma unroll
    for (int j = i; j < TA; ++j)
      if (i < S && j < S) {
        // one add per element per launch: deterministic fire-and-forget reduction
        float* dst = reinterpret_cast<float*>(p.part + (((size_t)kz * nbl + bl_index(i, j, S)) * p.G + g) *
                                                           (size_t)p.nchan + k);
        if (j == i) {
          atomicAdd(dst, auto_value(acc[i][j]).x);
        } else {
          atomicAdd(dst, acc[i][j].x);
          atomicAdd(dst + 1, acc[i][j].y);
        }
      }
}

// The same X step with the ring filled by the tensor memory accelerator: one
// 2-D tensor copy per stage (box: 128 channels x (kNB blocks x S stations))
// instead of 16-byte copies from every thread, so the bytes in flight are not
// limited by per-thread outstanding requests.  Thread 0 issues the copies; an
// mbarrier with a transaction count per ring slot signals arrival; every wait
// is bounded (timeout -> *err, the CTA stops issuing and returns).
constexpr long long kXDrainLimit = 1LL << 26;  // spins per wait while draining after an abort

__device__ __forceinline__ uint32_t xs_u32(const void* ptr) { return (uint32_t)__cvta_generic_to_shared(ptr); }

// Two threads per channel (256 per CTA): thread part 0 owns tile rows
// [0, SPLIT), part 1 rows [SPLIT, TA) -- about half the baselines each --
// so twice the warps share one ring of spectra.
constexpr int kXThreadsT = 2 * kXT;

// Bytes per spectrum value of each input kind: FP32 complex, FP16 complex
// (half2), E4M3 complex (two bytes, Re low).
// Blocks per ring stage: 2 of FP32, 4 of FP16, 8 of E4M3 values, so that a
// stage (and the bytes in flight per CTA) is the same size for every kind.
template <int IN> struct SpecElem {
  static constexpr int bytes = IN == 0 ? 8 : (IN == 1 ? 4 : 2);
  static constexpr int nb = kNB * 8 / bytes;
};

// One spectrum value from the ring as FP32 (the FP16 / E4M3 values carry
// X * 2^-sigma; the normalisation takes the 2^(2 sigma) back out).
template <int IN>
__device__ __forceinline__ float2 ring_value(const unsigned char* st, int idx) {
  if constexpr (IN == 0) {
    return reinterpret_cast<const float2*>(st)[idx];
  } else if constexpr (IN == 1) {
    return __half22float2(reinterpret_cast<const __half2*>(st)[idx]);
  } else {
    const __half2_raw h = __nv_cvt_fp8x2_to_halfraw2(reinterpret_cast<const __nv_fp8x2_storage_t*>(st)[idx], __NV_E4M3);
    return __half22float2(__half2(h));
  }
}

template <int TA, int IN>
__global__ void __launch_bounds__(kXThreadsT) k_xmac_tma(const __grid_constant__ CUtensorMap tmap, XParams p) {
  extern __shared__ __align__(1024) unsigned char xs_tma_raw[];
  const uint32_t raw = xs_u32(xs_tma_raw);
  constexpr int EB = SpecElem<IN>::bytes;
  constexpr int NB = SpecElem<IN>::nb;
  unsigned char* ring = xs_tma_raw + (((raw + 1023u) & ~1023u) - raw);  // [kStagesX][NB*S][kXT] values
  __shared__ __align__(8) uint64_t full[kStagesX];
  __shared__ int s_abort;
  const int tid = threadIdx.x;
  const int lane_ch = tid % kXT;
  const int part = tid / kXT;
  const int k0 = blockIdx.x * kXT;
  const int k = k0 + lane_ch;
  const int g = blockIdx.y;
  const int kz = blockIdx.z;
  const int S = p.S;
  const int b_lo = (int)((int64_t)p.CB * kz / p.KZ);
  const int b_hi = (int)((int64_t)p.CB * (kz + 1) / p.KZ);
  if (b_hi <= b_lo) return;
  const int nst = (b_hi - b_lo + NB - 1) / NB;
  const int stage_elems = NB * S * kXT;
  const uint32_t stage_bytes = (uint32_t)stage_elems * EB;
  if (tid == 0) {
    for (int i = 0; i < kStagesX; ++i) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(xs_u32(&full[i])));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_abort = 0;
  }
  __syncthreads();

  auto issue = [&](int q) {
    if (q >= nst) return;
    const int slot = q % kStagesX;
    const int row = (g * p.CB + b_lo + q * NB) * S;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(xs_u32(&full[slot])),
                 "r"(stage_bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            xs_u32(ring + (size_t)slot * stage_bytes)),
        "l"(reinterpret_cast<uint64_t>(&tmap)), "r"(2 * k0), "r"(row), "r"(xs_u32(&full[slot]))
        : "memory");
  };

  float2 acc[TA][TA];
#pragma unroll
  for (int i = 0; i < TA; ++i)
#pragma unroll
    for (int j = 0; j < TA; ++j) acc[i][j] = make_float2(0.f, 0.f);

  if (tid == 0)
    for (int q = 0; q < kStagesX - 1; ++q) issue(q);

  // rows [I0, I1) of this thread's part, compile-time per branch
  auto run = [&](auto I0c, auto I1c) {
    constexpr int I0 = decltype(I0c)::value, I1 = decltype(I1c)::value;
    int q = 0;
    for (; q < nst; ++q) {
      if (tid == 0) issue(q + kStagesX - 1);  // the slot of stage q-1, freed by the sync below
      const int slot = q % kStagesX;
      uint32_t ok = 0;
      for (long long it = 0; it < p.wait_limit && !ok; ++it) {
        asm volatile(
            "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
            : "=r"(ok)
            : "r"(xs_u32(&full[slot])), "r"((uint32_t)((q / kStagesX) & 1))
            : "memory");
        if ((it & 1023) == 1023 && s_abort) break;
      }
      if (!ok) s_abort = 1;
      __syncthreads();
      if (s_abort) break;
      const unsigned char* st = ring + (size_t)slot * stage_bytes;
#pragma unroll
      for (int bi = 0; bi < NB; ++bi) {
        if (b_lo + q * NB + bi >= b_hi) break;
        float2 a[TA];
#pragma unroll
        for (int i = I0; i < TA; ++i) a[i] = i < S ? ring_value<IN>(st, (bi * S + i) * kXT + lane_ch) : make_float2(0.f, 0.f);
#pragma unroll
        for (int i = I0; i < I1; ++i) {
          const float2 ar = rot_conj(a[i]);
#pragma unroll
          for (int j = i; j < TA; ++j)
            acc[i][j] = j == i ? cmac_auto(acc[i][j], a[i]) : cmac_conj(acc[i][j], a[i], ar, a[j]);
        }
      }
      __syncthreads();
    }
    if (s_abort) {
      // let the copies already issued land before the CTA's shared memory
      // goes away: stage q (whose wait gave up) and the ones issued after it
      if (tid == 0) {
        for (int r = q; r < q + kStagesX && r < nst; ++r) {
          const int slot = r % kStagesX;
          uint32_t ok = 0;
          for (long long it = 0; it < kXDrainLimit && !ok; ++it)
            asm volatile(
                "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
                : "=r"(ok)
                : "r"(xs_u32(&full[slot])), "r"((uint32_t)((r / kStagesX) & 1))
                : "memory");
        }
        if (p.err) atomicExch(p.err, 1);
      }
      return;
    }
    if (k >= p.nchan) return;
    const int nbl = nbl_of(S);
#pragma unroll
    for (int i = I0; i < I1; ++i)
#pragma unroll
      for (int j = i; j < TA; ++j)
        if (i < S && j < S) {
          float* dst = reinterpret_cast<float*>(p.part + (((size_t)kz * nbl + bl_index(i, j, S)) * p.G + g) *
                                                             (size_t)p.nchan + k);
          if (j == i) {
            atomicAdd(dst, auto_value(acc[i][j]).x);
          } else {
            atomicAdd(dst, acc[i][j].x);
            atomicAdd(dst + 1, acc[i][j].y);
          }
        }
  };
  constexpr int SPLIT = tri_split(TA, 2, 1);
  if (part == 0)
    run(std::integral_constant<int, 0>{}, std::integral_constant<int, SPLIT>{});
  else
    run(std::integral_constant<int, SPLIT>{}, std::integral_constant<int, TA>{});
}

static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(ptr);
    else
      cudaGetLastError();
  }
  return fn;
}

// The tensor map views the spectra as rows (stream, block, station) of 2 nchan
// scalars (Re, Im interleaved): FP32, FP16 or single bytes (E4M3 pairs); a
// stage is 2 x 128 scalars (128 channels, 256..1024 bytes, a multiple of 16)
// by NB * S rows (NB blocks per stage), from x = 2 k0 (a multiple of 256 scalars).
template <int TA, int IN>
static cudaError_t launch_tma_in(const XParams& p_in, cudaStream_t s, bool* used) {
  *used = false;
  XParams p = p_in;
  p.wait_limit = wait_limit();
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  constexpr int EB = SpecElem<IN>::bytes;
  constexpr int NB = SpecElem<IN>::nb;
  if (!enc || p.nchan < kXT || p.nchan % kXT || NB * p.S > 256) return cudaSuccess;
  CUtensorMap tm;
  cuuint64_t dims[2] = {(cuuint64_t)2 * p.nchan, (cuuint64_t)p.G * p.CB * p.S};
  cuuint64_t strides[1] = {(cuuint64_t)p.nchan * EB};
  cuuint32_t box[2] = {(cuuint32_t)(2 * kXT), (cuuint32_t)(NB * p.S)};
  cuuint32_t estr[2] = {1, 1};
  const CUtensorMapDataType dt =
      IN == 0 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : (IN == 1 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_UINT8);
  if (enc(&tm, dt, 2, const_cast<float2*>(p.spec), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
          CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return cudaSuccess;  // FP32: fall back to the cp.async ring
  const size_t smem = 1024 + (size_t)kStagesX * NB * p.S * kXT * EB;
  cudaError_t e = cudaFuncSetAttribute(k_xmac_tma<TA, IN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid((p.nchan + kXT - 1) / kXT, p.G, p.KZ);
  k_xmac_tma<TA, IN><<<grid, kXThreadsT, smem, s>>>(tm, p);
  *used = true;
  return cudaGetLastError();
}

template <int TA>
static cudaError_t launch_tma(const XParams& p, cudaStream_t s, bool* used) {
  if (p.in_kind == 1) return launch_tma_in<TA, 1>(p, s, used);
  if (p.in_kind == 2) return launch_tma_in<TA, 2>(p, s, used);
  return launch_tma_in<TA, 0>(p, s, used);
}

static int tile_for(int S) {
  if (S <= 2) return 2;
  if (S <= 4) return 4;
  if (S <= 6) return 6;
  if (S <= 8) return 8;
  if (S <= 10) return 10;
  if (S <= 12) return 12;
  return 8;
}

int xstage_kz(int CB, int S, int G, int nchan) {
  const int TA = tile_for(S);
  const int nt = (S + TA - 1) / TA;
  const long ctas = (long)((nchan + kXT - 1) / kXT) * G * (nt * (nt + 1) / 2);
  // about three waves of two CTAs per SM
  int kz = (int)((3L * 2 * 152 + ctas - 1) / ctas);
  const int by256 = (CB + 255) / 256;            // each partial sums <= 256 blocks
  if (kz < by256) kz = by256;
  if (kz > CB) kz = CB;
  if (kz < 1) kz = 1;
  return kz;
}

template <int TA>
static cudaError_t launch_ring(const XParams& p, cudaStream_t s) {
  bool used = false;
  cudaError_t te = launch_tma<TA>(p, s, &used);
  if (te != cudaSuccess || used) return te;
  if (p.in_kind != 0) return cudaErrorNotSupported;  // FP16 / E4M3 spectra: the TMA ring only
  const size_t smem = (size_t)kStagesX * kNB * p.S * kXT * sizeof(float2);
  cudaError_t e = cudaFuncSetAttribute(k_xmac_ring<TA>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid((p.nchan + kXT - 1) / kXT, p.G, p.KZ);
  k_xmac_ring<TA><<<grid, kXT, smem, s>>>(p);
  return cudaGetLastError();
}

template <int TA>
static cudaError_t launch_TA(const XParams& p, cudaStream_t s) {
  const int nt = (p.S + TA - 1) / TA;
  const int ntiles = (p.nchan + kXT - 1) / kXT;
  const size_t smem1 = (size_t)kStagesT * TA * kXT * sizeof(float2);
  cudaError_t e = cudaFuncSetAttribute(k_xmac<TA, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem1);
  if (e != cudaSuccess) return e;
  k_xmac<TA, true><<<dim3(nt * ntiles, p.G, p.KZ), 2 * kXT, smem1, s>>>(p, nt);
  if ((e = cudaGetLastError()) != cudaSuccess || nt == 1) return e;
  if constexpr (TA == 8) {  // only the 8-station tiling has off-diagonal tiles
    const size_t smem2 = 2 * smem1;
    e = cudaFuncSetAttribute(k_xmac<TA, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2);
    if (e != cudaSuccess) return e;
    k_xmac<TA, false><<<dim3(nt * (nt - 1) / 2 * ntiles, p.G, p.KZ), 2 * kXT, smem2, s>>>(p, nt);
    return cudaGetLastError();
  }
  return cudaErrorInvalidValue;
}

bool xstage_reduced_supported(int S, int nchan) {
  return S >= 1 && S <= 12 && SpecElem<2>::nb * S <= 256 && nchan >= kXT && nchan % kXT == 0 &&
         tensor_map_encoder() != nullptr;
}

cudaError_t launch_xstage(const XParams& p, cudaStream_t s) {
  if (p.CB <= 0) return cudaSuccess;
  if (p.in_kind != 0 && !xstage_reduced_supported(p.S, p.nchan)) return cudaErrorNotSupported;
  switch (tile_for(p.S)) {
    case 2: return launch_ring<2>(p, s);
    case 4: return launch_ring<4>(p, s);
    case 6: return launch_ring<6>(p, s);
    case 8: return p.S <= 8 ? launch_ring<8>(p, s) : launch_TA<8>(p, s);
    case 10: return launch_ring<10>(p, s);
    case 12: return launch_ring<12>(p, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace corr
