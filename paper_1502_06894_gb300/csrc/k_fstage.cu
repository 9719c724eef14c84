// k_fstage.cu -- the F step of the FX correlator (the paper, Abstract: each
// station's samples are Fourier transformed first, then cross-multiplied).
//
// One CTA takes one station and a few FFT blocks.  Per block it stages the
// packed 2-bit words of the delay-tracked window [b*N + n_b, +N) in shared
// memory once (all G streams of a station share one window), then each
// FFT group of T threads transforms one stream:
//
//   unpack   2-bit codes -> levels, two real samples per complex point through
//            one 16-entry table of level pairs (pre-halved, which absorbs the
//            split's 1/2), decoded straight into the registers of the first pass;
//   FFT      N real samples as an N/2-point complex FFT (even samples in the
//            real part, odd in the imaginary part), Stockham auto-sort passes
//            of radix 8/16/32 held in registers, shared memory between passes
//            (Stockham formulation as in Govindaraju et al., SC08);
//   split    X[k] = E[k] + W_N^k O[k], E = (Z[k] + conj Z[L-k])/2,
//            O = (Z[k] - conj Z[L-k])/(2i), k = 0..N/2-1 (Nyquist dropped);
//   rotate   X[k] *= exp(+2 pi i (phi + k*delta)), phi = frac(nu0 tau) and
//            delta = eps*fs/N from the FP64 delay kernel, FP32 within the block;
//   store    complex FP32 spectra [stream][block][station][channel], or for the
//            tensor-core X step complex FP16 times an exact power of two.
//
// Blocks that are not valid at this station (window outside the data, or no
// delay segment yet) store zeros, so they add nothing in the X step.
#include "k_fstage_impl.cuh"

#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

namespace corr {

unsigned long long current_context_id() {
  static PFN_cuCtxGetCurrent_v4000 get_cur = nullptr;
  static PFN_cuCtxGetId_v12000 get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 4000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_cur = reinterpret_cast<PFN_cuCtxGetCurrent_v4000>(p);
    p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<PFN_cuCtxGetId_v12000>(p);
    cudaGetLastError();
  });
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (!get_cur || !get_id || get_cur(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS) return 0;
  return id;
}

namespace {
std::mutex g_const_mu;
unsigned long long g_const_ctx[kMaxDevices];  // context the constants were loaded into, per device
}  // namespace

cudaError_t fstage_ensure_constants() {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  // a host-side lookup that also binds the device's context and loads this
  // module, so that the context id below is the one the kernels run in
  void* sym = nullptr;
  if ((e = cudaGetSymbolAddress(&sym, c_w32)) != cudaSuccess) return e;
  const unsigned long long id = current_context_id();
  std::lock_guard<std::mutex> lk(g_const_mu);
  // id 0 (no context id available): load once per device
  if (g_const_ctx[dev] != 0 && (id == 0 || g_const_ctx[dev] == id)) return cudaSuccess;
  if ((e = init_w32()) != cudaSuccess) return e;
  if ((e = fstage_pre_init_constants()) != cudaSuccess) return e;
  g_const_ctx[dev] = id ? id : ~0ull;
  return cudaSuccess;
}


// ---------------------------------------------------------------------------
// Tensor-core variant of the F step (FFT length N <= 2048): writes the FP16
// spectra directly as the X step's MMA operand tiles.  A tile holds one
// stream, one 64-block K range and a group of cpt channels: rows
// r = (channel-in-group * S + station) * 2 + {0: Re, 1: Im}, 128 rows x 64
// blocks of FP16, K-major with the 128-byte swizzle (16-byte chunk c of row r
// stored at chunk c ^ (r % 8)).  Two groups (W = 2 cpt channels) form one
// 32 KB pair that the X step fetches with a single bulk copy.
//
// One CTA takes one station and 8 consecutive blocks (one 16-byte K chunk).
// Per round its groups transform the 8 blocks of NGRP/8 streams, keep the
// FP16 spectra in shared memory, then all threads corner-turn them: for each
// channel and Re/Im the 8 blocks become one 16-byte store.  The packed
// samples are read straight from global memory (L1-cached across streams).
//
// FP8 (E4M3) tiles have the same geometry with one byte per value: a tile
// row holds 128 blocks, so a K tile spans 128 blocks and the 8 blocks of a
// CTA fill one half (8 bytes) of a 16-byte chunk.

template <int GC>
__device__ __forceinline__ void load_pair_g(const StationView& sv, int64_t rel, int G, int m, int j,
                                            uint32_t& c0, uint32_t& c1) {
  if constexpr (GC == 16) {
    const int64_t w = rel + 2 * m;  // one word per sample-time group
    uint32_t w0, w1;
    if ((rel & 1) == 0) {  // the pair is one aligned 64-bit load
      const uint2 x = __ldg(reinterpret_cast<const uint2*>(sv.words + w));
      w0 = x.x;
      w1 = x.y;
    } else {
      w0 = __ldg(&sv.words[w]);
      w1 = __ldg(&sv.words[w + 1]);
    }
    c0 = (w0 >> (2 * j)) & 3u;
    c1 = (w1 >> (2 * j)) & 3u;
  } else {
    const int64_t bit = 2 * ((rel + 2 * m) * G + j);
    c0 = (__ldg(&sv.words[bit >> 5]) >> (bit & 31)) & 3u;
    const int64_t bit1 = bit + 2 * G;
    c1 = (__ldg(&sv.words[bit1 >> 5]) >> (bit1 & 31)) & 3u;
  }
}

// Channels k (low half) and L - k (high half) of one block as one 8-byte
// slot: two FP16 complex values, or two E4M3 complex values in the low 4 bytes.
template <bool FP8>
__device__ __forceinline__ void put_pair(float2* slot, float2 a, float2 b, float scale) {
  if constexpr (FP8) {
    *reinterpret_cast<uint32_t*>(slot) = fp8x2(a.x * scale, a.y * scale) | (fp8x2(b.x * scale, b.y * scale) << 16);
  } else {
    const __half2 ha = __floats2half2_rn(a.x * scale, a.y * scale), hb = __floats2half2_rn(b.x * scale, b.y * scale);
    *reinterpret_cast<uint2*>(slot) = make_uint2(*reinterpret_cast<const uint32_t*>(&ha),
                                                 *reinterpret_cast<const uint32_t*>(&hb));
  }
}

// Byte address of row r's 16-byte chunk kc in the tile of (stream jo, channel ch, K tile kt).
__device__ __forceinline__ unsigned char* chunk_at(const TcTiles& o, int S, int s, int jo, int kt, int kc, int ch,
                                                   int reim) {
  const int sl = ch / o.W;
  const int cw = ch - sl * o.W;
  const int tg = cw / o.cpt;
  const int cl = cw - tg * o.cpt;
  const int r = (cl * S + s) * 2 + reim;
  unsigned char* tile = o.tiles + ((((size_t)jo * o.nslice + sl) * o.NKT + kt) * 2 + tg) * 16384;
  return tile + (r >> 3) * 1024 + (r & 7) * 128 + ((kc ^ (r & 7)) << 4);
}

// The FP16 values of channel ch (half h of each slot) in 8 consecutive
// blocks: one 16-byte chunk for Re and one for Im.
__device__ __forceinline__ void put_chunk16(const TcTiles& o, int S, int s, int jo, int kt, int kc, int ch,
                                            const uint2 (&w)[8], int h) {
  uint32_t re[4], im[4];
#pragma unroll
  for (int e = 0; e < 8; e += 2) {
    const uint32_t a = h ? w[e].y : w[e].x, b = h ? w[e + 1].y : w[e + 1].x;  // (Re, Im) as two halves
    re[e / 2] = __byte_perm(a, b, 0x5410);
    im[e / 2] = __byte_perm(a, b, 0x7632);
  }
  *reinterpret_cast<uint4*>(chunk_at(o, S, s, jo, kt, kc, ch, 0)) = make_uint4(re[0], re[1], re[2], re[3]);
  *reinterpret_cast<uint4*>(chunk_at(o, S, s, jo, kt, kc, ch, 1)) = make_uint4(im[0], im[1], im[2], im[3]);
}

// The same for E4M3: 8 blocks x (Re byte, Im byte) -> 8 Re bytes and 8 Im
// bytes, the half chunk khalf of the K range's 16-byte chunk.
__device__ __forceinline__ void put_chunk8(const TcTiles& o, int S, int s, int jo, int kt, int kc, int khalf, int ch,
                                           const uint32_t (&w)[8], int h) {
  uint32_t v[8];
#pragma unroll
  for (int e = 0; e < 8; ++e) v[e] = h ? (w[e] >> 16) : (w[e] & 0xffffu);
  const uint32_t r01 = __byte_perm(v[0], v[1], 0x0040), r23 = __byte_perm(v[2], v[3], 0x0040);
  const uint32_t r45 = __byte_perm(v[4], v[5], 0x0040), r67 = __byte_perm(v[6], v[7], 0x0040);
  const uint32_t i01 = __byte_perm(v[0], v[1], 0x0051), i23 = __byte_perm(v[2], v[3], 0x0051);
  const uint32_t i45 = __byte_perm(v[4], v[5], 0x0051), i67 = __byte_perm(v[6], v[7], 0x0051);
  *reinterpret_cast<uint2*>(chunk_at(o, S, s, jo, kt, kc, ch, 0) + khalf) =
      make_uint2(__byte_perm(r01, r23, 0x5410), __byte_perm(r45, r67, 0x5410));
  *reinterpret_cast<uint2*>(chunk_at(o, S, s, jo, kt, kc, ch, 1) + khalf) =
      make_uint2(__byte_perm(i01, i23, 0x5410), __byte_perm(i45, i67, 0x5410));
}

// Barrier of one team of 8 groups (8T threads, named barrier 1 + team) when
// there are several teams of whole warps, else of the CTA.
template <int T, int SPR>
__device__ __forceinline__ void tsync(int team) {
  if constexpr (SPR > 1 && (8 * T) % 32 == 0)
    asm volatile("bar.sync %0, %1;" ::"r"(team + 1), "r"(8 * T) : "memory");
  else
    __syncthreads();
}

template <int L, int GC, bool FP8>
__global__ void __launch_bounds__(Groups<L>::T * GroupsTC<L>::NGRP, MinBlocksTC<L>::v)
k_fstage_tc(FParams p, TcTiles o) {
  using P = Plan<L>;
  constexpr int T = P::T;
  constexpr int NGRP = GroupsTC<L>::NGRP;
  static_assert(NGRP >= 8 && NGRP % 8 == 0, "the tile writer needs 8 groups per stream");
  constexpr int SPR = NGRP / 8;  // teams: streams per round
  constexpr bool TEAMS = SPR > 1 && (8 * T) % 32 == 0;
  constexpr int BUF = kBufPad<L>();
  constexpr int R0 = P::R0;
  constexpr int PER0 = L / R0 / T;
  constexpr int HALF = L / 2;

  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* fbuf_all = reinterpret_cast<float2*>(smem_raw);
  __shared__ float2 s_lut16[16];
  __shared__ float2 s_tw[Tw<L>::size];
  fill_tables<L, LastRadix<L>::v>(s_lut16, s_tw, p);
  const int tid = threadIdx.x;
  const int grp = tid / T;
  const int t = tid - grp * T;
  const int team = grp / 8;
  float2* fbuf = fbuf_all + grp * BUF;
  const int s = blockIdx.y;
  const int G = GC ? GC : p.G;
  const StationView sv = p.st[s];
  const int blk = grp & 7;
  const int bb = blockIdx.x * 8 + blk;  // block within the chunk
  const bool present = bb < p.CB;
  const int d = p.blk0 + (present ? bb : 0);
  const bool valid = present && p.valid[(size_t)s * p.ld + d] != 0;
  const int64_t rel = valid ? p.start[(size_t)s * p.ld + d] - sv.sample0 : 0;
  const float delta = valid ? p.delta[(size_t)s * p.ld + d] : 0.f;
  constexpr int KB = FP8 ? 128 : 64;                  // blocks per K tile
  const int kt = (blockIdx.x * 8) / KB;
  const int kc = FP8 ? ((blockIdx.x & 15) >> 1) : (blockIdx.x & 7);  // 16-byte chunk of the K range
  const int khalf = FP8 ? (blockIdx.x & 1) * 8 : 0;   // byte offset of the FP8 half chunk
  __syncthreads();

  for (int r0 = 0; r0 < G; r0 += SPR) {
    const int j = r0 + team;
    const bool ok = valid && j < G;
    // the stream's fringe phase, loaded now so that its latency passes during the transform
    const float phi = ok ? p.phi[((size_t)s * p.nsub + j / p.npol) * p.ld + d] : 0.f;
    // ---- pass 0 from global memory (L1-cached across the stream rounds),
    //      skipped for blocks that are absent or not valid: their spectra
    //      are zeros ----
    if (ok) {
      float2 v[PER0][R0];
#pragma unroll
      for (int u = 0; u < PER0; ++u) {
        const int jj = t + u * T;
#pragma unroll
        for (int r = 0; r < R0; ++r) {
          const int m = jj + r * (L / R0);
          uint32_t c0, c1;
          load_pair_g<GC>(sv, rel, G, m, j, c0, c1);
          v[u][r] = s_lut16[c0 | (c1 << 2)];
        }
      }
#pragma unroll
      for (int u = 0; u < PER0; ++u) {
        const int jj = t + u * T;
        dft_reg<R0>(v[u]);
#pragma unroll
        for (int r = 0; r < R0; ++r) fbuf[padp<R0>(jj * R0 + r)] = v[u][r];
      }
      gsync<T>(grp);
      if constexpr (P::R1 > 1)
        stockham_pass<L, P::R1, P::R0, T, P::R0>(fbuf, t, grp, p.twN, Tw<L>::on ? s_tw : nullptr);
      if constexpr (P::R2 > 1) stockham_pass<L, P::R2, P::R0 * P::R1, T, P::R0>(fbuf, t, grp, p.twN);
    }

    // ---- real split + rotation; the FP16 (E4M3) values of channels k and
    //      L - k go into the float2 slot of Z[k]: only this thread reads
    //      that slot (and the one of Z[L - k]), so it writes without a
    //      barrier and holds nothing in registers ----
    constexpr int QF = HALF / T;  // k = t + qT < HALF for q < QF; k = HALF is thread 0's extra
    if (ok) {
      float2 z = cis_turns(fmaf((float)t, delta, phi));
      float2 y = cis_turns(fmaf((float)(L - t), delta, phi));
      float cm1, sn;
      walk_step((float)T * delta, cm1, sn);
      SplitTw<L, T> tw(s_tw, p.twN, t);
#pragma unroll 4
      for (int q = 0; q < QF; ++q) {
        const int k = t + q * T;
        float2 Xa, Xb;
        split_pair<L, R0>(fbuf, tw.get(s_tw, k), k, (L - k) & (L - 1), Xa, Xb);
        put_pair<FP8>(fbuf + padp<R0>(k), cmul(Xa, z), cmul(Xb, y), o.scale);
        z = walk(z, cm1, sn);
        y = walk(y, cm1, -sn);
        tw.next();
      }
      if (t == 0) {
        float2 Xa, Xb;
        split_pair<L, R0>(fbuf, make_float2(0.f, -1.f), HALF, HALF, Xa, Xb);
        put_pair<FP8>(fbuf + padp<R0>(HALF), cmul(Xa, z), make_float2(0.f, 0.f), o.scale);
      }
    } else {
      const float2 zero = make_float2(0.f, 0.f);
#pragma unroll 4
      for (int q = 0; q < QF; ++q) put_pair<FP8>(fbuf + padp<R0>(t + q * T), zero, zero, o.scale);
      if (t == 0) put_pair<FP8>(fbuf + padp<R0>(HALF), zero, zero, o.scale);
    }
    tsync<T, SPR>(team);

    // ---- corner turn: for each channel pair (c, L - c) the 8 blocks' slots
    //      become, per channel and Re/Im, one 16-byte chunk (FP8: 8 bytes);
    //      with teams each team turns its own stream ----
    const int ss0 = TEAMS ? team : 0;
    const int nss = TEAMS ? 1 : SPR;
    const int ttid = TEAMS ? tid - team * 8 * T : tid;
    const int tstride = TEAMS ? 8 * T : NGRP * T;
    for (int it = ttid; it < nss * (HALF + 1); it += tstride) {
      const int ss = ss0 + it / (HALF + 1);
      const int c = it - (ss - ss0) * (HALF + 1);
      const int jo = r0 + ss;
      if (jo >= G) continue;
      const float2* slot0 = fbuf_all + (size_t)(ss * 8) * BUF + padp<R0>(c);
      if constexpr (FP8) {
        uint32_t w[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) w[e] = *reinterpret_cast<const uint32_t*>(slot0 + e * BUF);
        put_chunk8(o, p.S, s, jo, kt, kc, khalf, c, w, 0);
        if (c != 0 && c != HALF) put_chunk8(o, p.S, s, jo, kt, kc, khalf, L - c, w, 1);
      } else {
        uint2 w[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) w[e] = *reinterpret_cast<const uint2*>(slot0 + e * BUF);
        put_chunk16(o, p.S, s, jo, kt, kc, c, w, 0);
        if (c != 0 && c != HALF) put_chunk16(o, p.S, s, jo, kt, kc, L - c, w, 1);
      }
    }
    tsync<T, SPR>(team);
  }
}

template <int L, int GC, bool FP8>
static cudaError_t launch_tc_LG(const FParams& p, const TcTiles& o, cudaStream_t st) {
  constexpr int T = Plan<L>::T;
  constexpr int NGRP = GroupsTC<L>::NGRP;
  const size_t smem = (size_t)NGRP * kBufPad<L>() * sizeof(float2);
  cudaError_t e =
      cudaFuncSetAttribute(k_fstage_tc<L, GC, FP8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  // whole K tiles: blocks at or beyond CB are written as zeros
  dim3 grid(o.NKT * (FP8 ? 16 : 8), p.S);
  k_fstage_tc<L, GC, FP8><<<grid, T * NGRP, smem, st>>>(p, o);
  return cudaGetLastError();
}

template <int L>
static cudaError_t launch_tc_L(const FParams& p, const TcTiles& o, cudaStream_t st) {
  if constexpr (GroupsTC<L>::NGRP % 8 == 0 && Plan<L>::T * GroupsTC<L>::NGRP <= 1024) {
    if (o.fp8) {
      if (p.G == 16) return launch_tc_LG<L, 16, true>(p, o, st);
      return launch_tc_LG<L, 0, true>(p, o, st);
    }
    if (p.G == 16) return launch_tc_LG<L, 16, false>(p, o, st);
    return launch_tc_LG<L, 0, false>(p, o, st);
  } else {
    return cudaErrorInvalidValue;
  }
}

bool fstage_tc_tiles_supported(int nchan) { return nchan >= 4 && nchan <= 1024; }

cudaError_t launch_fstage_tc(const FParams& p, const TcTiles& o, cudaStream_t s) {
  if (p.CB <= 0) return cudaSuccess;
  switch (p.nchan) {
    case 4: return launch_tc_L<4>(p, o, s);
    case 8: return launch_tc_L<8>(p, o, s);
    case 16: return launch_tc_L<16>(p, o, s);
    case 32: return launch_tc_L<32>(p, o, s);
    case 64: return launch_tc_L<64>(p, o, s);
    case 128: return launch_tc_L<128>(p, o, s);
    case 256: return launch_tc_L<256>(p, o, s);
    case 512: return launch_tc_L<512>(p, o, s);
    case 1024: return launch_tc_L<1024>(p, o, s);
    default: return cudaErrorInvalidValue;
  }
}

template <int L>
static cudaError_t launch_L(const FParams& p, cudaStream_t st) {
  if constexpr (L >= 256) {
    if (p.G == 16) return launch_LG<L, 16, false>(p, st);
    if (p.G == 32) return launch_LG<L, 32, false>(p, st);
  }
  return launch_LG<L, 0, false>(p, st);
}

bool fstage_supported(int nchan) {
  switch (nchan) {
    case 4: case 8: case 16: case 32: case 64: case 128: case 256: case 512:
    case 1024: case 2048: case 4096: case 8192:
      return true;
    default:
      return false;
  }
}

cudaError_t launch_fstage(const FParams& p, cudaStream_t s) {
  if (p.CB <= 0) return cudaSuccess;
  if (p.pre) return launch_fstage_pre(p, s);
  switch (p.nchan) {
    case 4: return launch_L<4>(p, s);
    case 8: return launch_L<8>(p, s);
    case 16: return launch_L<16>(p, s);
    case 32: return launch_L<32>(p, s);
    case 64: return launch_L<64>(p, s);
    case 128: return launch_L<128>(p, s);
    case 256: return launch_L<256>(p, s);
    case 512: return launch_L<512>(p, s);
    case 1024: return launch_L<1024>(p, s);
    case 2048: return launch_L<2048>(p, s);
    case 4096: return launch_L<4096>(p, s);
    case 8192: return launch_L<8192>(p, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace corr
