// k_fstage_impl.cuh -- the F-step kernel template shared by the real-transform
// (post-F rotation) and the pre-F rotation translation units.  Internal: each
// including translation unit gets its own copy of the radix-32 constant table
// (c_w32) and loads it through its own init function.
#pragma once
#include "corr_internal.cuh"

#include <cuda_fp8.h>

#include <algorithm>
#include <math.h>

namespace corr {

// Complex value -> two E4M3 bytes (Re in the low byte), round to nearest,
// saturating at +-448.
__device__ __forceinline__ uint32_t fp8x2(float re, float im) {
  return (uint32_t)__nv_cvt_float2_to_fp8x2(make_float2(re, im), __NV_SATFINITE, __NV_E4M3);
}


static __constant__ float2 c_w32[32];   // exp(-2 pi i m / 32)
static __constant__ float2 c_w32n[32];  // (-Im, Im) of the same, the second operand of a packed product

static cudaError_t init_w32() {
  float2 h[32], hn[32];
  for (int m = 0; m < 32; ++m) {
    double a = -2.0 * 3.14159265358979323846 * (double)m / 32.0;
    h[m] = make_float2((float)cos(a), (float)sin(a));
    hn[m] = make_float2(-h[m].y, h[m].y);
  }
  cudaError_t e = cudaMemcpyToSymbol(c_w32, h, sizeof(h));
  if (e != cudaSuccess) return e;
  return cudaMemcpyToSymbol(c_w32n, hn, sizeof(hn));
}

__host__ __device__ constexpr int ilog2c(int x) { return x <= 1 ? 0 : 1 + ilog2c(x >> 1); }
__host__ __device__ constexpr int bitrevc(int x, int bits) {
  int r = 0;
  for (int i = 0; i < bits; ++i) r |= ((x >> i) & 1) << (bits - 1 - i);
  return r;
}

// Complex arithmetic on packed FP32 pairs: one f32x2 instruction (add, mul
// or fma) computes both parts of a complex value with the rounding of two
// scalar instructions, which halves the instructions of the FFT butterflies
// and products (the F kernels are bound by instruction issue); the swapped
// and broadcast operands below are operand selections, not extra moves.
__device__ __forceinline__ float2 f2add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 f2sub(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ float2 f2mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 f2fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 swp(float2 a) { return make_float2(a.y, a.x); }
__device__ __forceinline__ float2 bc(float x) { return make_float2(x, x); }

// a b = (a.x b.x - a.y b.y, a.y b.x + a.x b.y) = a (b.x, b.x) + swap(a) (-b.y, b.y)
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return f2fma(swp(a), make_float2(-b.y, b.y), f2mul(a, bc(b.x)));
}
// a W_32^m, the second operand pair read ready-made from c_w32n
__device__ __forceinline__ float2 cmul_w32(float2 a, int m) {
  return f2fma(swp(a), c_w32n[m], f2mul(a, bc(c_w32[m].x)));
}

// Shared FFT buffers insert one padding element after every P elements (P =
// the first pass's radix): pass 0 stores each thread's P outputs contiguously,
// so without padding the threads of a half-warp would hit the same banks.
template <int P>
__device__ __forceinline__ int padp(int i) { return i + (i >> ilog2c(P)); }

// In-register DFT of R points (R <= 32): radix-2 decimation in frequency,
// natural-order input, output permuted back to natural order.  Butterflies
// with the twiddle -i rotate the difference by a swap and a sign pair.
template <int R>
__device__ __forceinline__ void dft_reg(float2 (&v)[R]) {
  constexpr int LOG = ilog2c(R);
#pragma unroll
  for (int st = 0; st < LOG; ++st) {
    const int half = R >> (st + 1);
#pragma unroll
    for (int i = 0; i < R; i += 2 * half) {
#pragma unroll
      for (int k = 0; k < half; ++k) {
        const float2 a = v[i + k], b = v[i + k + half];
        v[i + k] = f2add(a, b);
        const float2 d = f2sub(a, b);
        const int m = k * (32 / (2 * half));  // W_{2 half}^k = W_32^m
        if (m == 0)
          v[i + k + half] = d;
        else if (m == 8)
          v[i + k + half] = f2mul(swp(d), make_float2(1.f, -1.f));  // -i d
        else
          v[i + k + half] = cmul_w32(d, m);
      }
    }
  }
  float2 t[R];
#pragma unroll
  for (int r = 0; r < R; ++r) t[r] = v[bitrevc(r, LOG)];
#pragma unroll
  for (int r = 0; r < R; ++r) v[r] = t[r];
}

// Barrier of one FFT group of T threads (groups are T consecutive threads).
// Groups skip their transform independently (a block that is not valid), so
// a group never waits for lanes outside it: groups smaller than a warp sync
// on their own lane mask, larger ones on a named barrier of their own.
template <int T>
__device__ __forceinline__ void gsync(int grp) {
  if constexpr (T == 1) {
    // one thread: program order suffices
  } else if constexpr (T < 32) {
    const unsigned lane = threadIdx.x & 31u;
    __syncwarp(((1u << T) - 1u) << (lane & ~(unsigned)(T - 1)));
  } else if constexpr (T == 32) {
    __syncwarp();
  } else {
    asm volatile("bar.sync %0, %1;" ::"r"(grp + 1), "r"(T) : "memory");
  }
}

// v[r] *= W^{kr} for r = 1..R-1 from wp[i] = W^{k 2^i}.  r splits into its
// low LO bits a and its high bits b: W^{kr} = A[a] B[b] with A[a] = W^{ka}
// and B[b] = W^{k 2^LO b}, each the product of the wp of its bits.  Only the
// two short tables stay live (not one power per r), and every index is fixed
// at compile time, so all values stay in registers.
template <int N, int r = 1>
__device__ __forceinline__ void power_table(float2 (&A)[N], const float2* wp) {
  if constexpr (r < N) {
    constexpr int hb = ilog2c(r);
    if constexpr (r == (1 << hb))
      A[r] = wp[hb];
    else
      A[r] = cmul(A[r - (1 << hb)], wp[hb]);
    power_table<N, r + 1>(A, wp);
  }
}

template <int R, int NA, int NB, int r = 1>
__device__ __forceinline__ void apply_powers(float2 (&v)[R], const float2 (&A)[NA], const float2 (&B)[NB]) {
  if constexpr (r < R) {
    constexpr int a = r % NA, b = r / NA;
    if constexpr (a != 0 && b != 0)
      v[r] = cmul(cmul(v[r], A[a]), B[b]);
    else if constexpr (a != 0)
      v[r] = cmul(v[r], A[a]);
    else
      v[r] = cmul(v[r], B[b]);
    apply_powers<R, NA, NB, r + 1>(v, A, B);
  }
}

template <int R, int LOGR>
__device__ __forceinline__ void twiddle_products(float2 (&v)[R], const float2 (&wp)[LOGR]) {
  constexpr int LO = LOGR / 2;
  constexpr int NA = 1 << LO, NB = 1 << (LOGR - LO);
  float2 A[NA], B[NB];
  power_table<NA>(A, wp);
  power_table<NB>(B, wp + LO);
  apply_powers<R, NA, NB>(v, A, B);
}

// A later Stockham pass: read R points per butterfly group, twiddle, DFT,
// write back in place (all reads of the group finish before any write).
// W_{NS R}^{k r} = W_L^{k r L/(NS R)} = W_N^{TWS k r L/(NS R)} (TWS = N / L:
// 2 for the real transform packed into L = N/2 points, 1 for the complex
// N-point transform of the pre-F rotation).  For the last pass (NS R = L)
// from the shared table s_twl[r NS + k] when given; otherwise the powers
// W^k, W^2k, W^4k, ... come from the global table and W^{kr} is their
// product over the bits of r (at most log2 R - 1 multiplications deep),
// which keeps the memory pipeline, the bottleneck of the large transforms,
// to log2 R loads per butterfly group.  Those loads depend on the thread
// only, so they are issued first and their latency passes while the group
// reads its points and waits at the barrier.  With s_twp (transforms of
// 2048+ points) the powers come from a shared table [i][k] of the pass
// instead: consecutive k in consecutive words, read after the barrier.
template <int L, int R, int NS, int T, int P, int TWS = 2>
__device__ __forceinline__ void stockham_pass(float2* __restrict__ buf, int t, int grp,
                                              const float2* __restrict__ twN,
                                              const float2* __restrict__ s_twl = nullptr,
                                              const float2* __restrict__ s_twp = nullptr) {
  constexpr int GROUPS = L / R;
  constexpr int PER = GROUPS / T;
  constexpr int LOGR = ilog2c(R);
  static_assert(PER >= 1 && GROUPS % T == 0, "bad FFT plan");
  const bool tab = NS * R == L && s_twl != nullptr;
  const bool ptab = !tab && s_twp != nullptr;  // the powers from the shared table of this pass
  float2 wp[PER][LOGR];
  if (!tab && !ptab) {
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const int k = (t + u * T) & (NS - 1);
#pragma unroll
      for (int i = 0; i < LOGR; ++i) wp[u][i] = __ldg(&twN[TWS * k * (1 << i) * (L / (NS * R))]);
    }
  }
  float2 v[PER][R];
#pragma unroll
  for (int u = 0; u < PER; ++u) {
    const int j = t + u * T;
#pragma unroll
    for (int r = 0; r < R; ++r) v[u][r] = buf[padp<P>(j + r * GROUPS)];
  }
  gsync<T>(grp);
#pragma unroll
  for (int u = 0; u < PER; ++u) {
    const int j = t + u * T;
    const int k = j & (NS - 1);
    if (tab) {
#pragma unroll
      for (int r = 1; r < R; ++r) v[u][r] = cmul(v[u][r], s_twl[r * NS + k]);
    } else {
      if (ptab) {
#pragma unroll
        for (int i = 0; i < LOGR; ++i) wp[u][i] = s_twp[i * NS + k];
      }
      twiddle_products<R, LOGR>(v[u], wp[u]);
    }
    dft_reg<R>(v[u]);
    const int idxD = (j / NS) * NS * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) buf[padp<P>(idxD + r * NS)] = v[u][r];
  }
  gsync<T>(grp);
}

// FFT plans: L = N/2 complex points; radices R0*R1*R2 = L; T threads per FFT.
template <int L> struct Plan;
template <> struct Plan<4>    { static constexpr int R0 = 4,  R1 = 1,  R2 = 1, T = 1; };
template <> struct Plan<8>    { static constexpr int R0 = 8,  R1 = 1,  R2 = 1, T = 1; };
template <> struct Plan<16>   { static constexpr int R0 = 16, R1 = 1,  R2 = 1, T = 1; };
template <> struct Plan<32>   { static constexpr int R0 = 32, R1 = 1,  R2 = 1, T = 1; };
template <> struct Plan<64>   { static constexpr int R0 = 8,  R1 = 8,  R2 = 1, T = 8; };
template <> struct Plan<128>  { static constexpr int R0 = 16, R1 = 8,  R2 = 1, T = 8; };
template <> struct Plan<256>  { static constexpr int R0 = 16, R1 = 16, R2 = 1, T = 16; };
template <> struct Plan<512>  { static constexpr int R0 = 32, R1 = 16, R2 = 1, T = 16; };
template <> struct Plan<1024> { static constexpr int R0 = 32, R1 = 32, R2 = 1, T = 32; };
template <> struct Plan<2048> { static constexpr int R0 = 16, R1 = 16, R2 = 8, T = 128; };
template <> struct Plan<4096> { static constexpr int R0 = 16, R1 = 16, R2 = 16, T = 256; };
template <> struct Plan<8192> { static constexpr int R0 = 32, R1 = 16, R2 = 16, T = 256; };

template <int L> struct Groups {
  static constexpr int T = Plan<L>::T;
  // 256 threads per CTA (64 one-thread transforms for the smallest sizes);
  // 4096-point complex transforms (8192-sample blocks) run four independent
  // 256-thread transforms per CTA of 1024 threads, so that barriers stay
  // within a transform, four of them are in flight per SM and 32 warps hide
  // the latency of the twiddle loads
  static constexpr int NGRP = T == 1 ? 64 : (L == 4096 ? 3 : 256 / T);
};

// The tensor-core F step runs teams of 8 groups (one per block of its 8),
// one stream per team and round.
template <int L> struct GroupsTC {
  static constexpr int NGRP = Groups<L>::NGRP >= 8 ? Groups<L>::NGRP : 8;
};

template <int L> constexpr int kBufPad() { return L + L / Plan<L>::R0 + 1; }

// Shared tables for N <= 2048: the last Stockham pass's twiddles W_L^{k r}
// (L entries, [r][k]) and the real-split twiddles W_N^k for k <= L/2.
template <int L> struct Tw {
  static constexpr bool on = L >= 64 && L <= 1024;
  static constexpr int size = on ? L + L / 2 + 1 : 1;
};

// Fill the shared tables: s_lut16[c0 | c1 << 2] = (l[c0], l[c1]) / 2 (the
// halving takes the 1/2 of the real-FFT split into the input, exactly), and,
// when Tw<L>::on, the twiddle tables (last pass: NS = L / R_last).
template <int L, int RLAST, int TWS = 2>
__device__ __forceinline__ void fill_tables(float2* s_lut16, float2* s_tw, const FParams& p) {
  const int tid = threadIdx.x;
  if (tid < 16) {
    const float l[4] = {p.lut0, p.lut1, p.lut2, p.lut3};
    s_lut16[tid] = make_float2(0.5f * l[tid & 3], 0.5f * l[tid >> 2]);
  }
  if constexpr (Tw<L>::on) {
    constexpr int NS = L / RLAST;
    for (int e = tid; e < L; e += blockDim.x) {
      const int r = e / NS, k = e - r * NS;
      s_tw[e] = __ldg(&p.twN[TWS * k * r]);
    }
    for (int k = tid; k <= L / 2; k += blockDim.x) s_tw[L + k] = __ldg(&p.twN[k]);
  }
}

// Shared tables of the powers W^{k 2^i} (k < NS, i < log2 R) of the passes
// after the first, for transforms of 2048+ points: [i][k] per pass, the
// second pass's table after the first's.
template <int L> struct PassTw {
  static constexpr bool on = L >= 2048;
  static constexpr int n1 = Plan<L>::R1 > 1 ? ilog2c(Plan<L>::R1) * Plan<L>::R0 : 0;
  static constexpr int n2 = Plan<L>::R2 > 1 ? ilog2c(Plan<L>::R2) * Plan<L>::R0 * Plan<L>::R1 : 0;
  static constexpr int size = on ? n1 + n2 : 1;
};

template <int L, int R, int NS, int TWS>
__device__ __forceinline__ void fill_pass_table(float2* dst, const float2* __restrict__ twN) {
  constexpr int LOGR = ilog2c(R);
  for (int e = threadIdx.x; e < LOGR * NS; e += blockDim.x) {
    const int i = e / NS, k = e - i * NS;
    dst[e] = __ldg(&twN[TWS * k * (1 << i) * (L / (NS * R))]);
  }
}

template <int L, int TWS>
__device__ __forceinline__ void fill_pass_tables(float2* s_twp, const float2* __restrict__ twN) {
  if constexpr (PassTw<L>::on) {
    using P = Plan<L>;
    if constexpr (P::R1 > 1) fill_pass_table<L, P::R1, P::R0, TWS>(s_twp, twN);
    if constexpr (P::R2 > 1) fill_pass_table<L, P::R2, P::R0 * P::R1, TWS>(s_twp + PassTw<L>::n1, twN);
  }
}

template <int L> struct LastRadix {
  static constexpr int v = Plan<L>::R2 > 1 ? Plan<L>::R2 : (Plan<L>::R1 > 1 ? Plan<L>::R1 : Plan<L>::R0);
};

// ---- real split and rotation ----
// Channels k and L-k come from the same pair Z[k], Z[L-k] of the N/2-point
// transform:  X[k] = E + W O,  X[L-k] = conj(E - W O),  W = W_N^k.  Z is the
// transform of the halved samples, so E = Z[k] + conj Z[L-k] and
// O = -i (Z[k] - conj Z[L-k]) carry the split's factor 1/2.
template <int L, int R0>
__device__ __forceinline__ void split_pair(const float2* __restrict__ fbuf, float2 w, int k, int km, float2& Xa,
                                           float2& Xb) {
  const float2 Zk = fbuf[padp<R0>(k)];
  const float2 Zm = fbuf[padp<R0>(km)];
  const float2 pm = make_float2(1.f, -1.f), mp = make_float2(-1.f, 1.f);
  const float2 E = f2fma(Zm, pm, Zk);             // (Zk.x + Zm.x, Zk.y - Zm.y)
  const float2 Ec = f2fma(Zk, pm, Zm);            // conj E
  const float2 O = f2fma(swp(Zk), pm, swp(Zm));   // (Zk.y + Zm.y, Zm.x - Zk.x)
  const float2 WO = cmul(O, w);
  Xa = f2add(E, WO);
  Xb = f2fma(WO, mp, Ec);                         // (E.x - WO.x, WO.y - E.y)
}

// The split's twiddles W_N^k along a thread's channels k = t + qT: from the
// shared table for N <= 2048; above, W_N^t from the global table times
// W_N^{qT} by a walk (one product per channel instead of a global load
// whose latency the large transforms cannot hide; QF <= 16 steps add a few
// ulp).
template <int L, int T>
struct SplitTw {
  float2 w, step;
  __device__ __forceinline__ SplitTw(const float2* __restrict__ s_tw, const float2* __restrict__ twN, int t) {
    if constexpr (!Tw<L>::on) {
      w = __ldg(&twN[t]);
      step = __ldg(&twN[T]);
    }
  }
  __device__ __forceinline__ float2 get(const float2* __restrict__ s_tw, int k) const {
    if constexpr (Tw<L>::on) return s_tw[L + k];
    else return w;
  }
  __device__ __forceinline__ void next() {
    if constexpr (!Tw<L>::on) w = cmul(w, step);
  }
};

// The rotation exp(+2 pi i (phi + k delta)) along a thread's channels
// k = t + qT (and L - k): the first factor of each sequence comes from the
// fast sine/cosine of the argument reduced to [-pi, pi] (abs. error ~4e-7),
// later ones by a walk z <- z + z (e^{i theta} - 1), theta = +-2 pi T delta.
// |delta| <= 1/(2N) turns per channel (the fractional delay is at most half
// a sample), so |theta| <= pi T / N <= 0.2 and e^{i theta} - 1 comes from its
// Taylor series to theta^8 (remainder < 1e-12); written as an increment the
// walk has no systematic drift of |z| from rounding cos(theta).
__device__ __forceinline__ float2 cis_turns(float ph) {
  ph -= rintf(ph);
  float sn, cs;
  __sincosf(6.28318530717958648f * ph, &sn, &cs);
  return make_float2(cs, sn);
}

__device__ __forceinline__ void walk_step(float T_delta, float& cm1, float& sn) {
  const float th = 6.28318530717958648f * T_delta;
  const float t2 = th * th;
  // sin th = th (1 - th^2/3! + th^4/5! - th^6/7!)
  sn = th * fmaf(t2, fmaf(t2, fmaf(t2, -1.0f / 5040.0f, 1.0f / 120.0f), -1.0f / 6.0f), 1.0f);
  // cos th - 1 = th^2 (-1/2! + th^2/4! - th^4/6! + th^6/8!)
  cm1 = t2 * fmaf(t2, fmaf(t2, fmaf(t2, 1.0f / 40320.0f, -1.0f / 720.0f), 1.0f / 24.0f), -0.5f);
}

// z + z (cm1 + i sn) = (z + z cm1) + swap(z) (-sn, sn)
__device__ __forceinline__ float2 walk(float2 z, float cm1, float sn) {
  return f2fma(swp(z), make_float2(-sn, sn), f2fma(z, bc(cm1), z));
}

template <int OUT>
__device__ __forceinline__ void store_spec(void* out, size_t idx, float2 X, float scale) {
  if constexpr (OUT == 0) {
    reinterpret_cast<float2*>(out)[idx] = X;
  } else if constexpr (OUT == 1) {
    reinterpret_cast<__half2*>(out)[idx] = __floats2half2_rn(X.x * scale, X.y * scale);
  } else {
    reinterpret_cast<uint16_t*>(out)[idx] = (uint16_t)fp8x2(X.x * scale, X.y * scale);
  }
}

// Split, rotate and store the L/2 + 1 channel pairs of one transform; a
// block that is not valid stores zeros.
template <int L, int T, int R0, int OUT>
__device__ __forceinline__ void split_rotate_store(const float2* __restrict__ fbuf, const float2* __restrict__ s_tw,
                                                   const float2* __restrict__ twN, int t, bool ok, float phi,
                                                   float delta, void* out, size_t obase, float scale) {
  constexpr int HALF = L / 2;
  constexpr int QF = HALF / T;  // k = t + qT < HALF for q < QF; k = HALF is thread 0's extra
  const float2 zero = make_float2(0.f, 0.f);
  if (!ok) {
#pragma unroll 4
    for (int q = 0; q < QF; ++q) {
      const int k = t + q * T;
      store_spec<OUT>(out, obase + k, zero, scale);
      if (k != 0) store_spec<OUT>(out, obase + (L - k), zero, scale);
    }
    if (t == 0) store_spec<OUT>(out, obase + HALF, zero, scale);
    return;
  }
  float2 z = cis_turns(fmaf((float)t, delta, phi));
  float2 y = cis_turns(fmaf((float)(L - t), delta, phi));
  float cm1, sn;
  walk_step((float)T * delta, cm1, sn);
  SplitTw<L, T> tw(s_tw, twN, t);
#pragma unroll 4
  for (int q = 0; q < QF; ++q) {
    const int k = t + q * T;
    const int km = (L - k) & (L - 1);
    float2 Xa, Xb;
    split_pair<L, R0>(fbuf, tw.get(s_tw, k), k, km, Xa, Xb);
    store_spec<OUT>(out, obase + k, cmul(Xa, z), scale);
    if (k != 0) store_spec<OUT>(out, obase + km, cmul(Xb, y), scale);
    z = walk(z, cm1, sn);
    y = walk(y, cm1, -sn);
    tw.next();
  }
  if (t == 0) {  // k = HALF: X[HALF] = E + W_N^{N/4} O; z has walked to it
    float2 Xa, Xb;
    split_pair<L, R0>(fbuf, make_float2(0.f, -1.f), HALF, HALF, Xa, Xb);
    store_spec<OUT>(out, obase + HALF, cmul(Xa, z), scale);
  }
}

// Byte offset of the packed-word staging area after the NGRP FFT buffers,
// rounded up to 16 bytes for the 16-byte shared-memory stores.
template <int L>
constexpr size_t kWordsOffset(int NGRP) {
  return ((size_t)NGRP * kBufPad<L>() * sizeof(float2) + 15) & ~(size_t)15;
}

__host__ __device__ inline int wslot_words(int N, int G) {
  // window bits 2*N*G plus up to 31 bits of misalignment, up to 3 lead words
  // before the window, one word of shift (G = 16) and one spare word
  return (((2 * N * G + 31 + 31) >> 5) + 3 + 1 + 1 + 3) & ~3;
}

// Asynchronous global -> shared copies (LDGSTS) for the window staging.
__device__ __forceinline__ void cp_async16(void* sdst, const void* gsrc) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(sdst)),
               "l"(gsrc)
               : "memory");
}
__device__ __forceinline__ void cp_async8(void* sdst, const void* gsrc) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((uint32_t)__cvta_generic_to_shared(sdst)),
               "l"(gsrc)
               : "memory");
}
__device__ __forceinline__ void cp_async4(void* sdst, const void* gsrc) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((uint32_t)__cvta_generic_to_shared(sdst)),
               "l"(gsrc)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Stage the packed windows of `nslots` blocks (chunk blocks bb0...) into
// wbuf (slot stride wslot words) with asynchronous copies from device memory
// (plain loads from pinned host memory): 16-byte copies where the words lie
// inside the station's data, single words at its end.
// The copy of slot sl starts at the 16-byte aligned word a0 = w0 & ~3; with
// GC = 16 (one word per sample time) word w0 goes to an even index so that
// every sample pair is one aligned 64-bit load (odd leads are copied word by
// word, one word further on); with GC = 32 (two words per sample time, so
// the lead is 0 or 2) word w0 goes to a 16-byte boundary so that a sample
// pair is one aligned 16-byte load (a lead of 2 is copied in 8-byte pieces,
// two words further on).  s_ok / s_boff receive each slot's validity and the
// bit offset of its window from the slot's first word.
template <int N, int GC>
__device__ __forceinline__ void stage_windows(const FParams& p, const StationView& sv, int s, int G, int bb0,
                                              int nslots, uint32_t* wbuf, int wslot, int* s_ok, int* s_boff) {
  const int tid = threadIdx.x;
  for (int sl = 0; sl < nslots; ++sl) {
    const int d = p.blk0 + bb0 + sl;
    const bool ok = p.valid[(size_t)s * p.ld + d] != 0;
    int64_t w0 = 0;
    int boff = 0, nw = 0;
    if (ok) {
      const int64_t rel = p.start[(size_t)s * p.ld + d] - sv.sample0;
      const int64_t bit0 = 2 * rel * G;
      w0 = bit0 >> 5;
      boff = (int)(bit0 & 31);
      nw = (boff + 2 * N * G + 31) >> 5;
      if (w0 + nw > sv.nwords) nw = (int)(sv.nwords - w0);
    }
    const int lead = (int)(w0 & 3);
    // GC = 16: the window's first word at an even index; GC = 32 (lead 0
    // or 2): at a 16-byte boundary
    const int shift = (GC == 16) ? (lead & 1) : (GC == 32 ? ((4 - lead) & 3) : 0);
    uint32_t* dst = wbuf + sl * wslot + shift;
    const int64_t a0 = w0 - lead;
    const int ntot = nw + lead;
    const int nvec = ntot >> 2;
    if (sv.host) {
      // pinned host memory over the host link: plain 16-byte loads (they
      // keep more of the link's requests in flight than the async copies)
      const uint4* src4 = reinterpret_cast<const uint4*>(sv.words + a0);
      for (int q = tid; q < nvec; q += blockDim.x) {
        if (a0 + 4 * q + 4 <= sv.nwords) {
          const uint4 x = __ldg(src4 + q);
          if (shift) {
            dst[4 * q] = x.x;
            dst[4 * q + 1] = x.y;
            dst[4 * q + 2] = x.z;
            dst[4 * q + 3] = x.w;
          } else {
            reinterpret_cast<uint4*>(dst)[q] = x;
          }
        } else {
          for (int u = 0; u < 4; ++u)
            if (a0 + 4 * q + u < sv.nwords) dst[4 * q + u] = __ldg(&sv.words[a0 + 4 * q + u]);
        }
      }
      for (int q = 4 * nvec + tid; q < ntot; q += blockDim.x)
        if (a0 + q < sv.nwords) dst[q] = __ldg(&sv.words[a0 + q]);
    } else {
      for (int q = tid; q < nvec; q += blockDim.x) {
        if (a0 + 4 * q + 4 <= sv.nwords) {
          if (shift == 2) {
            cp_async8(dst + 4 * q, sv.words + a0 + 4 * q);
            cp_async8(dst + 4 * q + 2, sv.words + a0 + 4 * q + 2);
          } else if (shift) {
#pragma unroll
            for (int u = 0; u < 4; ++u) cp_async4(dst + 4 * q + u, sv.words + a0 + 4 * q + u);
          } else {
            cp_async16(dst + 4 * q, sv.words + a0 + 4 * q);
          }
        } else {
          for (int u = 0; u < 4; ++u)
            if (a0 + 4 * q + u < sv.nwords) cp_async4(dst + 4 * q + u, sv.words + a0 + 4 * q + u);
        }
      }
      for (int q = 4 * nvec + tid; q < ntot; q += blockDim.x)
        if (a0 + q < sv.nwords) cp_async4(dst + q, sv.words + a0 + q);
    }
    if (tid == 0) {
      s_ok[sl] = ok ? 1 : 0;
      s_boff[sl] = boff + 32 * (lead + shift);
    }
  }
}

// Compile-time stream count GC (0: runtime p.G).  With GC = 16 a sample-time
// group is exactly one 32-bit word (a sample pair is one aligned 64-bit
// load: the staging puts the window's first word at an even index); with
// GC = 32 it is two words.
template <int GC>
__device__ __forceinline__ void load_pair(const uint32_t* __restrict__ wsl, int boff, int G, int m, int j,
                                          uint32_t& c0, uint32_t& c1) {
  if constexpr (GC == 16) {
    // the staging put the window's first word at an even index
    const uint2 w = *reinterpret_cast<const uint2*>(wsl + 2 * m);
    c0 = (w.x >> (2 * j)) & 3u;
    c1 = (w.y >> (2 * j)) & 3u;
  } else if constexpr (GC == 32) {
    // the staging put the window's first word at a 16-byte boundary: the
    // four words of a sample pair are one aligned 16-byte load
    const uint4 w = *reinterpret_cast<const uint4*>(wsl + 4 * m);
    const bool hi = (j >> 4) != 0;
    c0 = ((hi ? w.y : w.x) >> (2 * (j & 15))) & 3u;
    c1 = ((hi ? w.w : w.z) >> (2 * (j & 15))) & 3u;
  } else {
    const int bit = boff + 2 * (2 * m * G + j);
    c0 = (wsl[bit >> 5] >> (bit & 31)) & 3u;
    const int bit1 = bit + 2 * G;
    c1 = (wsl[bit1 >> 5] >> (bit1 & 31)) & 3u;
  }
}

// CTAs per SM the register allocation must allow: larger FFTs run one group
// of 128-256 threads per FFT, so without a bound the compiler takes up to
// 255 registers and a single CTA fills the SM's register file.  (4096- and
// 8192-point transforms keep one CTA of 512 / 256 threads per SM: their
// buffers and staged windows fill shared memory anyway.)
template <int L> struct MinBlocks {
  static constexpr int v = (L >= 512 && L <= 1024) ? 2 : (L == 2048 ? 3 : 1);
};
// the tensor-core F step keeps its 8 groups' spectra in shared memory
template <int L> struct MinBlocksTC {
  static constexpr int v = Groups<L>::T * GroupsTC<L>::NGRP > 256 ? 1 : MinBlocks<L>::v;
};

// Row of the spectra output for stream j, chunk block bb, station s:
// [stream][block][station], or with both hands of two polarisations
// [subband][block][pol][station], which puts the 2S (station, pol) pairs of a
// subband side by side for the X step.
__device__ __forceinline__ size_t spec_row(const FParams& p, int j, int bb, int s) {
  if (p.cross) {
    const int sb = j / p.npol, pol = j - sb * p.npol;
    return ((size_t)(sb * p.CB + bb) * p.npol + pol) * p.S + s;
  }
  return ((size_t)j * p.CB + bb) * p.S + s;
}

// One sample of stream j: sample-time group m of the staged window.
template <int GC>
__device__ __forceinline__ uint32_t load_one(const uint32_t* __restrict__ wsl, int boff, int G, int m, int j) {
  if constexpr (GC == 16) {
    return (wsl[m] >> (2 * j)) & 3u;
  } else if constexpr (GC == 32) {
    return (wsl[2 * m + (j >> 4)] >> (2 * (j & 15))) & 3u;
  } else {
    const int bit = boff + 2 * (m * G + j);
    return (wsl[bit >> 5] >> (bit & 31)) & 3u;
  }
}

// Pre-F fringe rotation of sample m of a block: exp(+2 pi i phi_m) with
// phi_m = phi0 + m * delta_s (turns), phi0 = the phase at the block's first
// sample (FP64 on the host side of the delay kernel, reduced to [0, 1)) and
// delta_s = dhi + dlo the phase step per sample, split so that dhi has at
// most 10 significant bits: m * dhi is then exact in FP32 for m < 2^14, its
// whole turns drop out exactly, and phi_m carries an error of ~1e-7 turns.
__device__ __forceinline__ float2 prerot(int m, float phi0, float dhi, float dlo) {
  const float fm = (float)m;
  float a = fm * dhi;
  a -= rintf(a);
  return cis_turns(fmaf(fm, dlo, phi0) + a);
}

// Store of the pre-F path: channels k = 0..L/2-1 of the complex L-point
// transform, times the fractional-delay slope exp(+2 pi i k delta) (the
// fringe phase was applied before the transform), by the same walk as the
// post-F store.
template <int L, int T, int R0, int OUT>
__device__ __forceinline__ void rotate_store_pre(const float2* __restrict__ fbuf, int t, bool ok, float delta,
                                                 void* out, size_t obase, float scale) {
  constexpr int Q = (L / 2) / T;
  static_assert(Q >= 1 && (L / 2) % T == 0, "plan");
  if (!ok) {
#pragma unroll 4
    for (int q = 0; q < Q; ++q) store_spec<OUT>(out, obase + t + q * T, make_float2(0.f, 0.f), scale);
    return;
  }
  float2 z = cis_turns((float)t * delta);
  float cm1, sn;
  walk_step((float)T * delta, cm1, sn);
#pragma unroll 4
  for (int q = 0; q < Q; ++q) {
    const int k = t + q * T;
    store_spec<OUT>(out, obase + k, cmul(fbuf[padp<R0>(k)], z), scale);
    z = walk(z, cm1, sn);
  }
}

// The F kernel.  PRE = false: the N = 2L real samples of a block as an
// L-point complex transform (even/odd samples packed), real split, post-F
// rotation.  PRE = true: the N = L real samples rotated one by one by the
// fringe phase into an L-point complex transform, then the fractional-delay
// slope.
template <int L, int GC, bool PRE>
__global__ void __launch_bounds__(Groups<L>::T * Groups<L>::NGRP, MinBlocks<L>::v)
k_fstage(FParams p, int slots, int wslot, int nseq) {
  using P = Plan<L>;
  constexpr int T = P::T;
  constexpr int NGRP = Groups<L>::NGRP;
  constexpr int N = PRE ? L : 2 * L;   // real samples per block
  constexpr int TWS = PRE ? 1 : 2;     // twN holds W_N^m; the transform needs W_L
  constexpr int BUF = kBufPad<L>();
  constexpr int R0 = P::R0;
  constexpr int PER0 = L / R0 / T;
  static_assert(PER0 >= 1, "plan");

  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* fbuf_all = reinterpret_cast<float2*>(smem_raw);
  static_assert(kWordsOffset<L>(NGRP) % 16 == 0, "staging area must be 16-byte aligned");
  uint32_t* wbuf = reinterpret_cast<uint32_t*>(smem_raw + kWordsOffset<L>(NGRP));

  const int tid = threadIdx.x;
  const int grp = tid / T;
  const int t = tid - grp * T;
  float2* fbuf = fbuf_all + grp * BUF;
  const int s = blockIdx.y;
  const int G = GC ? GC : p.G;
  const StationView sv = p.st[s];

  // this CTA: nseq steps of `slots` blocks each, from chunk block `first`;
  // with nseq > 1 the windows of step it+1 are copied (asynchronously, into
  // the other half of a double buffer) while step it is transformed
  const int first = blockIdx.x * nseq * slots;
  if (first >= p.CB) return;

  __shared__ int s_boff[2][64];
  __shared__ int s_ok[2][64];
  __shared__ float2 s_lut16[16];
  __shared__ float2 s_tw[Tw<L>::size];
  __shared__ float2 s_twp[PassTw<L>::size];
  fill_tables<L, LastRadix<L>::v, TWS>(s_lut16, s_tw, p);
  fill_pass_tables<L, TWS>(s_twp, p.twN);

  stage_windows<N, GC>(p, sv, s, G, first, min(slots, p.CB - first), wbuf, wslot, s_ok[0], s_boff[0]);
  cp_async_commit();
  for (int it = 0; it < nseq; ++it) {
    const int bb0 = first + it * slots;
    if (bb0 >= p.CB) break;  // uniform over the CTA
    const int nslots = min(slots, p.CB - bb0);
    const int nb = it & 1;
    if (it + 1 < nseq && bb0 + slots < p.CB)
      stage_windows<N, GC>(p, sv, s, G, bb0 + slots, min(slots, p.CB - bb0 - slots), wbuf + (nb ^ 1) * slots * wslot,
                           wslot, s_ok[nb ^ 1], s_boff[nb ^ 1]);
    cp_async_commit();
    cp_async_wait<1>();  // this step's windows have landed (the next step's may still fly)
    __syncthreads();
    uint32_t* wcur = wbuf + nb * slots * wslot;

    const int ntasks = nslots * G;
    for (int base = 0; base < ntasks; base += NGRP) {
      const int task = base + grp;
      const bool active = task < ntasks;
      const int sl = active ? task / G : 0;
      const int j = active ? task - sl * G : 0;
      const bool ok = active && s_ok[nb][sl];
      const int boff = s_boff[nb][sl];
      // for GC = 16 / 32 the window starts on a word boundary: skip the lead
      // (and shift) words
      const uint32_t* wsl = wcur + sl * wslot + (GC ? (boff >> 5) : 0);
      const int d = p.blk0 + bb0 + sl;
      // the block's phase terms, loaded now so that their latency passes
      // during the transform
      const float delta = ok ? p.delta[(size_t)s * p.ld + d] : 0.f;
      const float phi = (ok && !PRE) ? p.phi[((size_t)s * p.nsub + j / p.npol) * p.ld + d] : 0.f;

      // ---- pass 0: unpack straight into registers (NS = 1, no twiddles);
      //      the transform of a block that is not valid is skipped ----
      if (ok) {
        float2 v[PER0][R0];
        if constexpr (PRE) {
          const size_t ps = ((size_t)s * p.nsub + j / p.npol) * p.ld + d;
          const float phi0 = p.phi[ps];
          const float2 dph = p.dphi[ps];
#pragma unroll
          for (int u = 0; u < PER0; ++u) {
            const int jj = t + u * T;
#pragma unroll
            for (int r = 0; r < R0; ++r) {
              const int m = jj + r * (L / R0);
              // s_lut16[c] = (l[c] / 2, l[0] / 2): twice its real part is level c
              const float lev = 2.0f * s_lut16[load_one<GC>(wsl, boff, G, m, j)].x;
              const float2 z = prerot(m, phi0, dph.x, dph.y);
              v[u][r] = f2mul(z, bc(lev));
            }
          }
        } else {
#pragma unroll
          for (int u = 0; u < PER0; ++u) {
            const int jj = t + u * T;
#pragma unroll
            for (int r = 0; r < R0; ++r) {
              const int m = jj + r * (L / R0);
              uint32_t c0, c1;
              load_pair<GC>(wsl, boff, G, m, j, c0, c1);
              v[u][r] = s_lut16[c0 | (c1 << 2)];
            }
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
          stockham_pass<L, P::R1, P::R0, T, P::R0, TWS>(fbuf, t, grp, p.twN, Tw<L>::on ? s_tw : nullptr,
                                                        PassTw<L>::on ? s_twp : nullptr);
        if constexpr (P::R2 > 1)
          stockham_pass<L, P::R2, P::R0 * P::R1, T, P::R0, TWS>(fbuf, t, grp, p.twN, nullptr,
                                                                PassTw<L>::on ? s_twp + PassTw<L>::n1 : nullptr);
      }

      // ---- store (real split and post-F rotation, or the pre-F path's slope) ----
      if (active) {
        const int bb = bb0 + sl;
        if constexpr (PRE) {
          constexpr int NCH = L / 2;
          const size_t obase = spec_row(p, j, bb, s) * (size_t)NCH;
          if (p.out_kind == 1)
            rotate_store_pre<L, T, R0, 1>(fbuf, t, ok, delta, p.out, obase, p.scale);
          else if (p.out_kind == 2)
            rotate_store_pre<L, T, R0, 2>(fbuf, t, ok, delta, p.out, obase, p.scale);
          else
            rotate_store_pre<L, T, R0, 0>(fbuf, t, ok, delta, p.out, obase, p.scale);
        } else {
          const size_t obase = spec_row(p, j, bb, s) * (size_t)L;
          if (p.out_kind == 1)
            split_rotate_store<L, T, R0, 1>(fbuf, s_tw, p.twN, t, ok, phi, delta, p.out, obase, p.scale);
          else if (p.out_kind == 2)
            split_rotate_store<L, T, R0, 2>(fbuf, s_tw, p.twN, t, ok, phi, delta, p.out, obase, p.scale);
          else
            split_rotate_store<L, T, R0, 0>(fbuf, s_tw, p.twN, t, ok, phi, delta, p.out, obase, p.scale);
        }
      }
      gsync<T>(grp);
    }
    __syncthreads();  // every read of this step's windows is done before they are overwritten
  }
}

template <int L, int GC, bool PRE>
static cudaError_t launch_LG(const FParams& p, cudaStream_t st) {
  constexpr int T = Plan<L>::T;
  constexpr int NGRP = Groups<L>::NGRP;
  const int N = PRE ? L : 2 * L;
  int slots = NGRP / p.G;
  if (slots < 1) slots = 1;
  if (slots > 64) slots = 64;
  const int wslot = wslot_words(N, p.G);
  const size_t one = kWordsOffset<L>(NGRP) + (size_t)slots * wslot * sizeof(uint32_t);
  const size_t two = one + (size_t)slots * wslot * sizeof(uint32_t);
  // Several steps per CTA (tables filled once, the next windows copied while
  // the current ones are transformed) when the double buffer still lets the
  // kernel keep its CTAs per SM and the grid stays at 8+ waves of them.
  static int sm_count = 0;
  if (!sm_count) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sm_count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      sm_count = 152;
  }
  const int64_t steps = (int64_t)((p.CB + slots - 1) / slots) * p.S;
  int nseq = 1;
  if ((size_t)MinBlocks<L>::v * (two + sizeof(float2) * (Tw<L>::size + PassTw<L>::size) + 1024) <= 227 * 1024)
    nseq = (int)std::max<int64_t>(1, std::min<int64_t>(4, steps / ((int64_t)8 * MinBlocks<L>::v * sm_count)));
  const size_t smem = nseq > 1 ? two : one;
  if (smem + sizeof(float2) * (Tw<L>::size + PassTw<L>::size) + 1024 > 227 * 1024) return cudaErrorInvalidConfiguration;
  cudaError_t e = cudaFuncSetAttribute(k_fstage<L, GC, PRE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int per_cta = slots * nseq;
  dim3 grid((p.CB + per_cta - 1) / per_cta, p.S);
  k_fstage<L, GC, PRE><<<grid, T * NGRP, smem, st>>>(p, slots, wslot, nseq);
  return cudaGetLastError();
}

}  // namespace corr
