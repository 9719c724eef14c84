// k_xmma.cu -- the X step on the 5th-generation tensor cores (tcgen05), FP16
// or FP8 (E4M3) inputs with FP32 accumulation in tensor memory (TMEM).
//
// For one stream g and channel k the X step is a Hermitian outer product over
// the FFT blocks b of an integration:  V_ab = sum_b X_a[b] conj(X_b[b]).  With
// rows R = (Re X_0, Im X_0, Re X_1, Im X_1, ...) (2S rows, K = blocks) the real
// product P = R R^T holds every term:
//     V_ab = (P[2a][2b] + P[2a+1][2b+1]) + i (P[2a+1][2b] - P[2a][2b+1]).
// Several channels share one 128-row tile (cpt = floor(64/S) channels of 2S
// rows), so one M=N=128 MMA (K=16 of kind::f16, or K=32 of kind::f8f6f4)
// serves them all; the products across different channels are computed and
// discarded.  A = B = the same shared-memory tile.
//
// Operand tiles: 128 rows x 128 bytes, K-major with the 128-byte swizzle:
// 64 blocks of FP16 or 128 blocks of E4M3 per row, written by the F step
// (directly, or by the corner turns k_tiles / k_tiles8 from FP16 / FP8
// spectra); the X kernel k_xmma2 streams them with bulk copies into shared
// memory, issues the MMAs into TMEM accumulators and adds V_ab into FP32
// partial sums in global memory.  Both element types advance 32 bytes of a
// row per MMA, so the shared-memory descriptors are the same.
// Every wait on an mbarrier is bounded; on timeout the CTA sets *err, stops
// issuing work, waits (again bounded) for the bulk copies and MMAs it has in
// flight, frees its TMEM and returns.
#include "corr_internal.cuh"

#include <cuda_fp16.h>

#include <algorithm>
#include <atomic>

namespace corr {

namespace {

constexpr int kKT = 64;            // blocks per K tile (64 FP16 = one 128-byte swizzle row)
constexpr int kTileBytes = 128 * kKT * 2;  // one 128-row operand tile
constexpr long long kWaitLimit = 1LL << 26;  // spins before an mbarrier wait gives up (default)
constexpr long long kDrainLimit = 1LL << 26; // spins per wait while draining after an abort

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// K-major operand tile, 128-byte swizzle: element (row r, k) of a 128 x 64
// FP16 tile lives at byte (r/8)*1024 + (r%8)*128 + ((k/8) ^ (r%8))*16 + (k%8)*2.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  return ((uint64_t)((saddr >> 4) & 0x3FFF)) | (1ull << 16) /* LBO (unused for SW128 K-major) */ |
         (64ull << 32) /* SBO = 1024 B between 8-row groups */ | (1ull << 46) /* descriptor version */ |
         (2ull << 61) /* 128-byte swizzle */;
}

// Instruction descriptor: D FP32 (bits 4-5 = 1), A and B format code 0 (FP16
// for kind::f16, E4M3 for kind::f8f6f4), both K-major, N = M = 128.
constexpr uint32_t kIdesc = (1u << 4) | ((128u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ void mma_f16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t acc) {
  asm volatile(
      "{ .reg .pred p; setp.ne.b32 p, %4, 0; tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p; }" ::"r"(
          tmem_d),
      "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(acc));
}

__device__ __forceinline__ void mma_f8(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t acc) {
  asm volatile(
      "{ .reg .pred p; setp.ne.b32 p, %4, 0; tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p; }" ::"r"(
          tmem_d),
      "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
        "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
        "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

}  // namespace

// ---------------------------------------------------------------------------
// k_xmma2: the X step from ready-made operand tiles (written by the tensor-core
// F step), in the warp-specialised form of a Blackwell GEMM:
//   warp 4, lane 0  producer + MMA issuer: one 32 KB cp.async.bulk per K tile
//                   into a 6-stage ring (mbarrier with transaction count), then
//                   8 MMAs (2 channel groups x 4 K steps) into one of two
//                   256-column TMEM accumulators, tcgen05.commit to free the
//                   stage / publish the accumulator;
//   warps 0-3       epilogue: TMEM -> registers, Re/Im lane shuffle, V_ab into
//                   the partial sums, then release the accumulator.
// Every wait is bounded; a timeout sets *err and makes all roles stop.
namespace {

constexpr int kStages2 = 6;
constexpr int kPairBytes = 2 * kTileBytes;  // two channel-group tiles per K tile

__device__ __forceinline__ bool mbar_wait_abort(uint64_t* bar, uint32_t parity, volatile int* abort_flag,
                                                long long limit) {
  uint32_t ok = 0;
  for (long long it = 0; it < limit; ++it) {
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    if (ok) return true;
    if ((it & 1023) == 1023 && *abort_flag) return false;
  }
  return false;
}

// A bounded wait that ignores the abort flag: used after an abort, for the
// CTA's own copies and MMAs, which finish by themselves.
__device__ __forceinline__ bool mbar_drain_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok = 0;
  for (long long it = 0; it < kDrainLimit; ++it) {
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

// Named barrier 1 over the 128 epilogue threads, returning the OR of v.
__device__ __forceinline__ bool bar_or_128(bool v) {
  uint32_t r;
  asm volatile(
      "{ .reg .pred p, q; setp.ne.u32 q, %1, 0; bar.red.or.pred p, 1, 128, q; selp.u32 %0, 1, 0, p; }"
      : "=r"(r)
      : "r"((uint32_t)v)
      : "memory");
  return r != 0;
}

}  // namespace

template <bool FP8>
__global__ void __launch_bounds__(160, 1) k_xmma2(XTC2Params p, int nitems) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  unsigned char* ring = smem_raw + (((raw + 1023u) & ~1023u) - raw);  // [kStages2][32 KB]
  __shared__ __align__(8) uint64_t s_full[kStages2], s_empty[kStages2], s_acc_full[2], s_acc_empty[2], s_drain;
  __shared__ uint32_t s_taddr;
  __shared__ volatile int s_abort;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int S = p.S, cpt = p.cpt, W = p.W, nchan = p.nchan, NKT = p.NKT;
  const int nbl = nbl_of(S);
  const int rows_valid = 2 * S * cpt;

  if (tid == 0) {
    for (int i = 0; i < kStages2; ++i) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&s_full[i])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&s_empty[i])));
    }
    for (int i = 0; i < 2; ++i) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&s_acc_full[i])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 128;" ::"r"(smem_u32(&s_acc_empty[i])));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&s_drain)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_abort = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(&s_taddr)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t taddr = s_taddr;

  // items of this CTA: blockIdx.x, blockIdx.x + gridDim.x, ...; each has NKT K tiles
  const int my_items = nitems > (int)blockIdx.x ? (nitems - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  const int my_tiles = my_items * NKT;

  if (warp == 4) {
    if (lane == 0) {
      const long long lim = p.wait_limit;
      int loaded = 0;  // tiles whose bulk copy has been issued
      int landed = 0;  // tiles whose copy has been seen complete
      bool mma_issued = false;
      auto load = [&](int u) {
        const int n = u / NKT, kt = u - n * NKT;
        const int item = blockIdx.x + n * gridDim.x;  // = g * nslice + sl
        const int st = u % kStages2;
        const unsigned char* src = p.tiles + ((size_t)item * NKT + kt) * kPairBytes;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(&s_full[st])),
                     "r"(kPairBytes)
                     : "memory");
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                smem_u32(ring + st * kPairBytes)),
            "l"(src), "r"(kPairBytes), "r"(smem_u32(&s_full[st]))
            : "memory");
        loaded = u + 1;
      };
      for (int u = 0; u < kStages2 && u < my_tiles; ++u) load(u);
      for (int u = 0; u < my_tiles && !s_abort; ++u) {
        const int n = u / NKT, kt = u - n * NKT;
        const int st = u % kStages2;
        const int ab = n & 1;
        if (!mbar_wait_abort(&s_full[st], (u / kStages2) & 1, &s_abort, lim)) { s_abort = 1; break; }
        landed = u + 1;
        if (kt == 0 && n >= 2 && !mbar_wait_abort(&s_acc_empty[ab], ((n - 2) >> 1) & 1, &s_abort, lim)) {
          s_abort = 1;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
        for (int grp = 0; grp < 2; ++grp) {
          const uint64_t d0 = sw128_desc(smem_u32(ring + st * kPairBytes + grp * kTileBytes));
#pragma unroll
          for (int ks = 0; ks < 4; ++ks) {
            // 32 bytes of each row per MMA: K = 16 FP16 or K = 32 E4M3 values
            if constexpr (FP8)
              mma_f8(taddr + ab * 256 + grp * 128, d0 + 2ull * ks, d0 + 2ull * ks, (kt > 0 || ks > 0) ? 1u : 0u);
            else
              mma_f16(taddr + ab * 256 + grp * 128, d0 + 2ull * ks, d0 + 2ull * ks, (kt > 0 || ks > 0) ? 1u : 0u);
          }
        }
        mma_issued = true;
        mma_commit(&s_empty[st]);
        if (kt == NKT - 1) mma_commit(&s_acc_full[ab]);
        // refill the stage of the previous tile (its MMAs have had a whole
        // iteration to finish), not the one just issued
        if (u >= 1) {
          const int pv = u - 1;
          const int nxt = pv + kStages2;
          if (nxt < my_tiles) {
            if (!mbar_wait_abort(&s_empty[pv % kStages2], (pv / kStages2) & 1, &s_abort, lim)) { s_abort = 1; break; }
            load(nxt);
          }
        }
      }
      if (s_abort) {
        // drain before the CTA's shared memory and TMEM go away: every bulk
        // copy issued lands (each tile's full barrier completes its phase),
        // and every MMA issued completes (a commit of all prior tcgen05
        // operations of this thread to a barrier of its own)
        for (int t = landed; t < loaded; ++t) mbar_drain_wait(&s_full[t % kStages2], (t / kStages2) & 1);
        if (mma_issued) {
          mma_commit(&s_drain);
          mbar_drain_wait(&s_drain, 0);
        }
      }
    }
  } else {
    // ---- epilogue warps 0..3: TMEM lane quadrant = warp ----
    // V_ab of the item's W channels go to a shared stage [channel][baseline]
    // (every element written once), then out to the partial sums as
    // coalesced 16-byte vector reductions: the item's partials are one
    // contiguous run of W * nbl complex values.
    float2* stage = reinterpret_cast<float2*>(ring + kStages2 * kPairBytes);
    const int r = warp * 32 + lane;
    const bool re_lane = ((lane & 1) == 0) && r < rows_valid;
    const int a = (r >> 1) % S;
    const int cl = (r >> 1) / S;
    int rlast = warp * 32 + 31;
    if (rlast > rows_valid - 1) rlast = rows_valid - 1;
    const int cmin = (warp * 32) / (2 * S), cmax = rlast / (2 * S);
    const int q0 = (2 * S * cmin) / 32, q1 = (warp * 32 < rows_valid) ? (2 * S * (cmax + 1) - 1) / 32 : -1;
    for (int n = 0; n < my_items; ++n) {
      const int ab = n & 1;
      const bool timed_out = !mbar_wait_abort(&s_acc_full[ab], (n >> 1) & 1, &s_abort, p.wait_limit);
      // the four epilogue warps share named barriers below, so they stop
      // together: a barrier OR over their timeouts and the abort flag
      if (bar_or_128(timed_out || s_abort)) {
        s_abort = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int item = blockIdx.x + n * gridDim.x;
      const int g = item / p.nslice;
      const int c0 = (item - g * p.nslice) * W;
      const int nch = min(W, nchan - c0);
#pragma unroll 1
      for (int grp = 0; grp < 2; ++grp) {
        const int kc = grp * cpt + cl;  // channel within the item
        const bool mine = re_lane && c0 + kc < nchan;
        float2* srow = stage + (size_t)kc * nbl;
#pragma unroll 1
        for (int q = q0; q <= q1; ++q) {
          uint32_t v[32];
          tmem_ld32(taddr + ((uint32_t)(warp * 32) << 16) + ab * 256 + grp * 128 + q * 32, v);
          // column pair jj = q*16 + i holds (channel clj, station b) = divmod(jj, S)
          int clj = (q * 16) / S;
          int b = q * 16 - clj * S;
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            const float m0 = __uint_as_float(v[2 * i]), m1 = __uint_as_float(v[2 * i + 1]);
            const float n0 = __shfl_down_sync(0xffffffffu, m0, 1);
            const float n1 = __shfl_down_sync(0xffffffffu, m1, 1);
            if (mine && clj == cl && b >= a) srow[bl_index(a, b, S)] = make_float2(m0 + n1, n0 - m1);
            if (++b == S) {
              b = 0;
              ++clj;
            }
          }
        }
      }
      // the accumulator has been read: hand it back to the MMA issuer
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&s_acc_empty[ab])) : "memory");
      asm volatile("bar.sync 1, 128;" ::: "memory");  // stage complete
      // each partial-sum element gets exactly one add per launch, so the
      // fire-and-forget reductions keep the sums deterministic
      float* dst = reinterpret_cast<float*>(p.part + ((size_t)g * nchan + c0) * nbl);
      const float* src = reinterpret_cast<const float*>(stage);
      const int nf = nch * nbl * 2;  // a multiple of 4: nch is even
      for (int e = 4 * r; e < nf; e += 4 * 128) {
        const float4 x = *reinterpret_cast<const float4*>(src + e);
        asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(dst + e), "f"(x.x), "f"(x.y), "f"(x.z),
                     "f"(x.w)
                     : "memory");
      }
      asm volatile("bar.sync 1, 128;" ::: "memory");  // stage free for the next item
    }
  }

  __syncthreads();
  if (tid == 0 && s_abort) atomicExch(p.err, 1);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(taddr));
}

namespace {
std::atomic<long long> g_wait_limit{kWaitLimit};
}

void set_wait_limit(long long spins) { g_wait_limit.store(spins < 0 ? kWaitLimit : spins); }
long long wait_limit() { return g_wait_limit.load(); }

cudaError_t launch_xtc2(const XTC2Params& p_in, int sm_count, cudaStream_t s) {
  XTC2Params p = p_in;
  p.wait_limit = wait_limit();
  const int nitems = p.G * p.nslice;
  if (nitems <= 0 || p.NKT <= 0) return cudaSuccess;
  // the bulk-copy ring plus the epilogue's stage of W * nbl complex values
  // (at most 64 (S + 1) of them: 33,280 bytes at 64 stations)
  const size_t smem = 1024 + (size_t)kStages2 * kPairBytes + (size_t)p.W * nbl_of(p.S) * sizeof(float2);
  if (p.W % 2 || p.nchan % 2 || smem > 227 * 1024) return cudaErrorInvalidValue;
  const int grid = nitems < sm_count ? nitems : sm_count;
  if (p.fp8) {
    cudaError_t e = cudaFuncSetAttribute(k_xmma2<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_xmma2<true><<<grid, 160, smem, s>>>(p, nitems);
  } else {
    cudaError_t e = cudaFuncSetAttribute(k_xmma2<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_xmma2<false><<<grid, 160, smem, s>>>(p, nitems);
  }
  return cudaGetLastError();
}

// Corner turn of FP16 spectra into operand tiles, for FFT lengths at which
// the F step cannot hold 8 blocks of spectra in shared memory.  One CTA takes
// CH channels of one stream and one 64-block K tile:
//   stage   the spectra of all stations and the tile's 64 blocks, split into
//           Re and Im rows of 64 FP16 values (one 128-byte tile row each, in
//           block order; rows 144 bytes apart so that neighbouring channels
//           fall in different banks), from 16-byte reads of 4 channels, four
//           blocks per thread;
//   write   8 threads per row, one 16-byte chunk each, to the chunk's swizzled
//           place: every tile row is written as one whole 128-byte line.
// Blocks at or beyond cb are written as zeros (the MMA reads whole K tiles).
constexpr int kTurnRow = 144;  // bytes per staged row (128 bytes of values + 16 bytes of padding)

// Write phase of both corner turns: 8 threads per staged row, one 16-byte
// chunk each, to the chunk's swizzled place, so every tile row is written as
// one whole 128-byte line.
__device__ __forceinline__ void write_staged_rows(const unsigned char* turn_raw, const TcTiles& o, int S, int nch,
                                                  int CH, int c0, int kt, int jo) {
  // a thread keeps one (channel, 16-byte chunk) pair and runs over the 2S
  // rows (station, Re/Im) of that channel: the tile coordinates of the
  // channel are divided out once per thread, not once per chunk
  const int per = CH * 8;                  // (channel, chunk) pairs; CH * 8 divides the 256 threads
  const int comb = threadIdx.x & (per - 1);
  const int c = comb >> 3, kc = comb & 7;
  if (c >= nch) return;  // no barrier follows in any caller
  const int k = c0 + c;
  const int sl = k / o.W;
  const int cw = k - sl * o.W;
  const int tg = cw / o.cpt;
  const int cl = cw - tg * o.cpt;
  unsigned char* tile = o.tiles + ((((size_t)jo * o.nslice + sl) * o.NKT + kt) * 2 + tg) * 16384;
  for (int rs = threadIdx.x / per; rs < 2 * S; rs += blockDim.x / per) {
    const int ri = rs >= S ? 1 : 0;
    const int s = rs - ri * S;
    const uint4 v = *reinterpret_cast<const uint4*>(turn_raw + ((size_t)rs * CH + c) * kTurnRow + kc * 16);
    const int r = (cl * S + s) * 2 + ri;
    *reinterpret_cast<uint4*>(tile + (r >> 3) * 1024 + (r & 7) * 128 + ((kc ^ (r & 7)) << 4)) = v;
  }
}

__global__ void __launch_bounds__(256) k_tiles(const __half2* __restrict__ spec, TcTiles o, int CB, int cb, int S,
                                               int nchan, int CH) {
  extern __shared__ __align__(16) unsigned char turn_raw[];  // [Re/Im][S][CH] rows of kTurnRow bytes
  const int c0 = blockIdx.x * CH;
  const int kt = blockIdx.y;
  const int jo = blockIdx.z;
  const int nch = min(CH, nchan - c0);
  const int tid = threadIdx.x;
  // staging: a thread takes 4 channels x 4 consecutive blocks of one station
  // (four 16-byte loads in flight), and stores per channel the 4 Re and the
  // 4 Im values as one 8-byte piece of each row.  Threads run over blocks
  // fastest, so a half-warp fills 64-byte runs of two rows that sit in
  // different banks (rows 4 apart are 576 bytes apart).
  const int lcv = CH == 16 ? 2 : (CH == 8 ? 1 : 0);  // CV = CH / 4 = 2^lcv
  const int nstage = S * 2 * (8 << lcv);
  // the loads of two items are issued before either item's stores, so
  // eight 16-byte loads are in flight per thread (the kernel is bound by the
  // latency of its HBM reads)
  auto decode = [&](int i, int& c, int& sb, int& b0) {
    const int b4 = i & 7;
    const int j = i >> 3;
    c = 4 * (j & ((1 << lcv) - 1));
    const int rest = j >> lcv;
    sb = rest >> 1;
    b0 = (rest & 1) * 32 + b4 * 4;
  };
  for (int i0 = tid; i0 < nstage; i0 += 2 * blockDim.x) {
    uint4 v[2][4];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int i = i0 + h * blockDim.x;
      int c, sb, b0;
      decode(i, c, sb, b0);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int bg = kt * 64 + b0 + u;
        v[h][u] = make_uint4(0u, 0u, 0u, 0u);
        if (i < nstage && c < nch && bg < cb)
          v[h][u] = __ldg(reinterpret_cast<const uint4*>(spec + (((size_t)jo * CB + bg) * S + sb) * (size_t)nchan + c0 + c));
      }
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int i = i0 + h * blockDim.x;
      if (i >= nstage) break;
      int c, sb, b0;
      decode(i, c, sb, b0);
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        uint32_t w[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) w[u] = e == 0 ? v[h][u].x : e == 1 ? v[h][u].y : e == 2 ? v[h][u].z : v[h][u].w;
        const uint2 re = make_uint2((w[0] & 0xFFFFu) | (w[1] << 16), (w[2] & 0xFFFFu) | (w[3] << 16));
        const uint2 im = make_uint2((w[0] >> 16) | (w[1] & 0xFFFF0000u), (w[2] >> 16) | (w[3] & 0xFFFF0000u));
        *reinterpret_cast<uint2*>(turn_raw + ((size_t)sb * CH + c + e) * kTurnRow + 2 * b0) = re;
        *reinterpret_cast<uint2*>(turn_raw + ((size_t)(S + sb) * CH + c + e) * kTurnRow + 2 * b0) = im;
      }
    }
  }
  __syncthreads();
  write_staged_rows(turn_raw, o, S, nch, CH, c0, kt, jo);
}

// FP8 corner turn: the same, for E4M3 spectra (two bytes per channel: Re,
// Im) and 128-block K tiles.  A thread takes 8 channels (one 16-byte read) x
// 4 consecutive blocks of one station and stores per channel 4 Re and 4 Im
// bytes; threads run over blocks fastest, so a warp fills one whole 128-byte
// staged row.
__global__ void __launch_bounds__(256) k_tiles8(const uint16_t* __restrict__ spec8, TcTiles o, int CB, int cb,
                                                int S, int nchan, int CH) {
  extern __shared__ __align__(16) unsigned char turn_raw[];  // [Re/Im][S][CH] rows of kTurnRow bytes
  const int c0 = blockIdx.x * CH;
  const int kt = blockIdx.y;
  const int jo = blockIdx.z;
  const int nch = min(CH, nchan - c0);
  const int tid = threadIdx.x;
  const int lcv = CH == 16 ? 1 : 0;  // CV = CH / 8 = 2^lcv
  const int nstage = S * (32 << lcv);
  // two items' loads before either item's stores (eight 16-byte loads in flight)
  auto decode = [&](int i, int& b4, int& c, int& sb) {
    b4 = i & 31;
    const int j = i >> 5;
    c = 8 * (j & ((1 << lcv) - 1));
    sb = j >> lcv;
  };
  for (int i0 = tid; i0 < nstage; i0 += 2 * blockDim.x) {
    uint4 v[2][4];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int i = i0 + h * blockDim.x;
      int b4, c, sb;
      decode(i, b4, c, sb);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int bg = kt * 128 + 4 * b4 + u;
        v[h][u] = make_uint4(0u, 0u, 0u, 0u);
        if (i < nstage && c < nch && bg < cb)
          v[h][u] = __ldg(reinterpret_cast<const uint4*>(spec8 + (((size_t)jo * CB + bg) * S + sb) * (size_t)nchan + c0 + c));
      }
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int i = i0 + h * blockDim.x;
      if (i >= nstage) break;
      int b4, c, sb;
      decode(i, b4, c, sb);
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        uint32_t w[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int q = e >> 1;
          w[u] = q == 0 ? v[h][u].x : q == 1 ? v[h][u].y : q == 2 ? v[h][u].z : v[h][u].w;
        }
        // channel e sits in bytes 0,1 (even e) or 2,3 (odd e) of its word
        const uint32_t sre = (e & 1) ? 0x0062u : 0x0040u, sim = (e & 1) ? 0x0073u : 0x0051u;
        const uint32_t re = __byte_perm(__byte_perm(w[0], w[1], sre), __byte_perm(w[2], w[3], sre), 0x5410);
        const uint32_t im = __byte_perm(__byte_perm(w[0], w[1], sim), __byte_perm(w[2], w[3], sim), 0x5410);
        *reinterpret_cast<uint32_t*>(turn_raw + ((size_t)sb * CH + c + e) * kTurnRow + 4 * b4) = re;
        *reinterpret_cast<uint32_t*>(turn_raw + ((size_t)(S + sb) * CH + c + e) * kTurnRow + 4 * b4) = im;
      }
    }
  }
  __syncthreads();
  write_staged_rows(turn_raw, o, S, nch, CH, c0, kt, jo);
}

// Persistent FP16 corner turn: each CTA walks work items (channel group,
// K tile, stream); item i+1's spectra are copied with cp.async into the
// other half of a double-buffered raw stage ([station][block][CH] as 16-byte
// pieces of 4 channels) while item i is rearranged from the raw stage into
// the staged tile rows and written, so that the HBM reads of one item
// overlap the rearrangement and the writes of the one before.
__global__ void __launch_bounds__(256, 1) k_tiles_p(const __half2* __restrict__ spec, TcTiles o, int CB, int cb,
                                                   int S, int nchan, int CH, int ngroups, int nitems) {
  extern __shared__ __align__(16) unsigned char tp_raw[];
  const int PPR = CH / 4;                                  // 16-byte pieces per (station, block)
  const int raw_pieces = S * 64 * PPR;                     // per raw buffer
  uint4* raw = reinterpret_cast<uint4*>(tp_raw);           // [2][S][64][PPR]
  unsigned char* turn_raw = tp_raw + (size_t)2 * raw_pieces * 16;  // [Re/Im][S][CH] rows of kTurnRow bytes
  const uint32_t raw_s = (uint32_t)__cvta_generic_to_shared(raw);
  const int tid = threadIdx.x;
  auto decode_item = [&](int it, int& c0, int& kt, int& jo) {
    const int cg = it % ngroups;
    const int rest = it / ngroups;
    c0 = cg * CH;
    kt = rest % o.NKT;
    jo = rest / o.NKT;
  };
  auto issue = [&](int it, int buf) {
    if (it < nitems) {
      int c0, kt, jo;
      decode_item(it, c0, kt, jo);
      for (int e = tid; e < raw_pieces; e += blockDim.x) {
        const int q = e % PPR;
        const int row = e / PPR;                           // sb * 64 + block
        const int blk = row & 63;
        const int sb = row >> 6;
        const int bg = kt * 64 + blk;
        const int c = c0 + 4 * q;
        const bool in = bg < cb && c < nchan;
        const __half2* src = spec + (((size_t)jo * CB + (in ? bg : 0)) * S + sb) * (size_t)nchan + (in ? c : 0);
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(raw_s + (uint32_t)((buf * raw_pieces + e) * 16)),
                     "l"(src), "r"(in ? 16 : 0));
      }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  const int lcv = CH == 16 ? 2 : (CH == 8 ? 1 : 0);        // CV = CH / 4 = 2^lcv
  const int nstage = S * 2 * (8 << lcv);
  int buf = 0;
  issue(blockIdx.x, 0);
  for (int it = blockIdx.x; it < nitems; it += gridDim.x, buf ^= 1) {
    issue(it + gridDim.x, buf ^ 1);
    asm volatile("cp.async.wait_group 1;" ::: "memory");
    __syncthreads();  // raw[buf] has landed; the previous item's rows are written
    int c0, kt, jo;
    decode_item(it, c0, kt, jo);
    const int nch = min(CH, nchan - c0);
    const uint4* rb = raw + buf * raw_pieces;
    for (int i = tid; i < nstage; i += blockDim.x) {
      const int b4 = i & 7;
      const int j = i >> 3;
      const int c = 4 * (j & ((1 << lcv) - 1));
      const int rest = j >> lcv;
      const int sb = rest >> 1;
      const int b0 = (rest & 1) * 32 + b4 * 4;
      uint4 v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) v[u] = rb[(sb * 64 + b0 + u) * PPR + (c >> 2)];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        uint32_t w[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) w[u] = e == 0 ? v[u].x : e == 1 ? v[u].y : e == 2 ? v[u].z : v[u].w;
        const uint2 re = make_uint2((w[0] & 0xFFFFu) | (w[1] << 16), (w[2] & 0xFFFFu) | (w[3] << 16));
        const uint2 im = make_uint2((w[0] >> 16) | (w[1] & 0xFFFF0000u), (w[2] >> 16) | (w[3] & 0xFFFF0000u));
        *reinterpret_cast<uint2*>(turn_raw + ((size_t)sb * CH + c + e) * kTurnRow + 2 * b0) = re;
        *reinterpret_cast<uint2*>(turn_raw + ((size_t)(S + sb) * CH + c + e) * kTurnRow + 2 * b0) = im;
      }
    }
    __syncthreads();
    // the rows of this item's channels; threads of channels beyond nch skip
    // the writes (no barrier inside)
    write_staged_rows(turn_raw, o, S, nch, CH, c0, kt, jo);
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
}

cudaError_t launch_tiles(const __half2* spec, const TcTiles& o, int CB, int cb, int S, int G, int nchan,
                         cudaStream_t s) {
  if (cb <= 0) return cudaSuccess;
  {
    // persistent form: raw double buffer + staged rows = 800 S CH bytes <= 210 KB
    int CH = 16;
    while (CH > 4 && (size_t)800 * S * CH > 210 * 1024) CH /= 2;
    const size_t smem = (size_t)800 * S * CH;
    if (smem <= 210 * 1024 && nchan >= 4) {
      static int sm_count = 0;
      if (!sm_count) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sm_count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
          sm_count = 152;
      }
      const int ngroups = (nchan + CH - 1) / CH;
      const int nitems = ngroups * o.NKT * G;
      cudaError_t e = cudaFuncSetAttribute(k_tiles_p, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      k_tiles_p<<<std::min(nitems, sm_count), 256, smem, s>>>(spec, o, CB, cb, S, nchan, CH, ngroups, nitems);
      return cudaGetLastError();
    }
  }
  // channels per CTA: the staged rows stay within about 100 KB
  int CH = 16;
  while (CH > 4 && (size_t)2 * S * CH * kTurnRow > 100 * 1024) CH /= 2;
  const size_t smem = (size_t)2 * S * CH * kTurnRow;
  cudaError_t e = cudaFuncSetAttribute(k_tiles, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid((nchan + CH - 1) / CH, o.NKT, G);
  k_tiles<<<grid, 256, smem, s>>>(spec, o, CB, cb, S, nchan, CH);
  return cudaGetLastError();
}

cudaError_t launch_tiles8(const uint16_t* spec8, const TcTiles& o, int CB, int cb, int S, int G, int nchan,
                          cudaStream_t s) {
  if (cb <= 0) return cudaSuccess;
  if (nchan % 8) return cudaErrorInvalidValue;
  int CH = 16;
  while (CH > 8 && (size_t)2 * S * CH * kTurnRow > 110 * 1024) CH /= 2;
  const size_t smem = (size_t)2 * S * CH * kTurnRow;
  cudaError_t e = cudaFuncSetAttribute(k_tiles8, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid((nchan + CH - 1) / CH, o.NKT, G);
  k_tiles8<<<grid, 256, smem, s>>>(spec8, o, CB, cb, S, nchan, CH);
  return cudaGetLastError();
}

int xtc_cpt(int S) { return S <= 64 ? 64 / S : 0; }

}  // namespace corr
