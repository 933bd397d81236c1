// Spectral derivative along one axis (Sec. 2.2: the derivatives are taken
// with FFTs) as a dense contraction on the 5th-generation tensor cores, for
// the FP64 form.
//
// Along axis j the FFT derivative d_j f = IFFT_j[i (k + theta/L) FFT_j[f]] is
// one linear map applied to every line of n points: the circulant n x n
// complex matrix
//     D[m][q] = d[(m - q) mod n],  d[r] = (i / n) sum_a kappa_a e^{2 pi i a r / n},
// kappa_a = (2 pi a' + theta) / L with a' = a or a - n (FFT order; the Nyquist
// wavenumber kept, as in the line passes).  On the interleaved (re, im)
// storage it is the real 2n x 2n matrix
//     Dr[2m + c'][2q + c] = [[Re D, -Im D], [Im D, Re D]][c'][c],
// so one pass over nb arrays is OUT = LINES Dr^T with one row per line
// (nb G / n rows, K = N = 2n, padded to NC = a multiple of 16).  Both
// operands are cut into six base-256 digits (oz_digits.cuh), each line scaled
// by its own exponent and each row of Dr by its own; the 21 digit products of
// weight g = s + t <= 5 are summed in FP32 in TMEM: weights 0-3 exactly, one
// accumulator each (per K value |G_g| <= (g + 3) 2^14, K <= 64, so every sum
// stays an integer below 2^24), weights 4 and 5 together in a fifth, the
// weight-5 products taken with the operator's digits times 2^-8 (exact in
// bf16); its FP32 rounding, at most K 2^-24 of a sum below 2^23 at weight
// 2^-32, is about 2^-49 of the largest term.  The sums are combined in a
// 64-bit integer, rounded once to FP64 and scaled by the two exponents.  The
// error is that rounding plus the truncated digit expansion, about 2^-48 of
// the line's and the row's largest values.
//
// Persistent kernel, one CTA per SM, 128 lines per tile:
//   warps 0-7   producers: warp w takes lines 16 w .. 16 w + 15 of the tile,
//               lanes 0-15 the first half of each line's points and lanes
//               16-31 the second; a thread loads its half line at once, the
//               pair agrees on the line's exponent by one shuffle, and each
//               writes its digits into a ring stage in the canonical
//               no-swizzle K-major layout (8-row x 16-byte core matrices),
//               fences the writes for the tensor core's proxy and arrives;
//   warp 8      owns TMEM (two accumulator sets of 5 x NC fp32 columns, so
//               the MMAs of one tile run while the epilogue drains the
//               previous one; one set when 5 NC > 256); one lane issues
//               tcgen05.mma (M = 128, N = NC, K = 16) for every digit pair;
//   warps 9-16  epilogue: two warps per TMEM lane quadrant, half the columns
//               each, in blocks of 8 columns; they combine the groups into
//               64-bit integers, round, scale and store the (re, im) pairs at
//               the line's points (in place is allowed: tiles own disjoint
//               lines), then hand the accumulator set back.
// The operator's digits, computed once per context on the host in long
// double, stay in shared memory for the whole launch.  Every mbarrier wait is
// bounded; a timeout sets SKY_ETIMEOUT, the kernel waits (bounded) for the
// MMAs it issued, frees TMEM and returns.
#include <cmath>
#include <cstring>
#include <vector>

#include "oz_digits.cuh"
#include "oz_gemm.cuh"

namespace sky {
namespace ozd {

using namespace ozdig;
using tc::fence_after;
using tc::fence_before;
using tc::idesc_bf16;
using tc::mbar_init;
using tc::mbar_wait;
using tc::mma_bf16;
using tc::mma_commit;
using tc::smem_u32;

constexpr int S = 6;               // digits per operand (FP64 inputs)
constexpr int BM = 128;            // lines per tile (MMA M)
constexpr int kProd = 8, kEpi = 8;   // producer warps: two threads per line
constexpr int THREADS = 32 * (kProd + 1 + kEpi);
constexpr int kSmemMax = 232448;   // dynamic shared memory opt-in limit per CTA
constexpr int kBars = 24;
constexpr int NG = 5;              // TMEM groups: weights 0, 1, 2, 3 and {4, 5}

__host__ __device__ constexpr int nc_of(int n) { return ((2 * n + 15) / 16) * 16; }

// Operators of an axis: the derivative, the forward and the inverse DFT.
constexpr int kOpDeriv = 0, kOpFwd = 1, kOpInv = 2;
// Producer input: the lines of src, or the residual src - eps psi (src = h psi).
constexpr int kInPlain = 0, kInResidual = 1;
// Epilogue output: the product; times P[point] scale; or psi - w[point] times it.
constexpr int kOutPlain = 0, kOutScaleP = 1, kOutUpdate = 2;

template <int N>
struct Shape {
  static constexpr int NC = nc_of(N);          // K and output columns (reals), padded
  static constexpr int TILE_A = BM * NC * 2;   // one digit of a tile of lines
  static constexpr int STAGE = S * TILE_A;
  static constexpr int TILE_B = NC * NC * 2;   // one digit of the operator
  static constexpr int OPB = 2 * S * TILE_B;   // its digits, then the digits times 2^-8
  static constexpr int NBUF = NG * NC <= 256 ? 2 : 1;   // TMEM accumulator sets
  static constexpr int AUX = NC * 4 + 2 * BM * 4 + kBars * 8 + 16;
  static constexpr int H0 = ((N / 2 + 3) / 4) * 4;             // points of a line's first half
  // staging of the next tile's half lines (one 16-byte slot per point and
  // producer thread) when it fits beside one ring stage
  static constexpr int STG_BYTES = H0 * kProd * 32 * 16;
  static constexpr bool PREFETCH = STAGE + OPB + AUX + STG_BYTES + 1024 <= kSmemMax;
  static constexpr int STG = PREFETCH ? STG_BYTES : 0;
  static constexpr int STAGES = (2 * STAGE + OPB + AUX + STG + 1024 <= kSmemMax) ? 2 : 1;
  static constexpr int SMEM = STAGES * STAGE + OPB + AUX + STG + 1024;
  static constexpr int HALF = NC / 2;          // columns per epilogue warp
  static_assert(NG * NC <= 512, "TMEM columns");
  static_assert(SMEM <= kSmemMax, "shared memory");
  static_assert(HALF % 8 == 0, "TMEM load blocks of 8 columns");
  static_assert(NC <= 64, "int32 bounds of the group combination");
};

// Byte offset of element (r, k) of a K-major bf16 tile with nc columns in the
// canonical no-swizzle layout: 8 x 8 core matrices of 128 contiguous bytes,
// 128 bytes apart along K, 16 nc bytes apart along the rows.
__host__ __device__ constexpr int cm_off(int r, int k, int nc) {
  return (r >> 3) * (nc * 16) + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2;
}
// Shared-memory matrix descriptor of that layout: leading byte offset 128
// (core matrices along K), stride byte offset 16 nc (8-row groups), version 1,
// layout type 0 (no swizzle).
__device__ __forceinline__ uint64_t ns_desc(uint32_t saddr, int nc) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)(128 >> 4) << 16) |
         ((uint64_t)((nc * 16) >> 4) << 32) | (1ull << 46);
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
// 16-byte asynchronous copy global -> shared (zero fill when !valid).
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, bool valid) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src),
               "r"(valid ? 16 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// The six balanced base-256 digits of the signed integer Y = +-round(|x|
// 2^{48 - E}) (|Y| <= 2^48), as floats: adding 128 to each of the five lower
// byte positions (0x8080808080) turns every lower byte, minus 128, into a
// digit in [-128, 127], with the carries propagated by the addition; the top
// digit is the rest, an arithmetic shift (|digit 0| <= 256).  All exact in bf16.
__device__ __forceinline__ void digits6f(double x, int E, float* d) {
  long long Y = (long long)fixed_of<6>(x, E);
  if (sign_of(x)) Y = -Y;
  const long long Z = Y + 0x8080808080LL;
  const unsigned lo = (unsigned)Z, hi = (unsigned)((unsigned long long)Z >> 32);
  auto f = [](int v) { return __int_as_float(0x4B400000 + v) - 12582912.0f; };   // exact, |v| < 2^22
  d[5] = f((int)(lo & 255u) - 128);
  d[4] = f((int)((lo >> 8) & 255u) - 128);
  d[3] = f((int)((lo >> 16) & 255u) - 128);
  d[2] = f((int)(lo >> 24) - 128);
  d[1] = f((int)(hi & 255u) - 128);
  d[0] = f((int)(Z >> 40));
}
__device__ __forceinline__ unsigned bf16x2(float lo, float hi) {   // lo in the low half
  unsigned r;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
  return r;
}
// v 2^sc rounded to the nearest double (halfway cases away from zero), by
// integer operations on the bit pattern; results outside the normal range go
// through ldexp.
__device__ __forceinline__ double scaled_double(long long v, int sc) {
  if (v == 0) return 0.0;
  const unsigned long long neg = v < 0 ? (1ull << 63) : 0ull;
  const unsigned long long u = v < 0 ? (unsigned long long)(-v) : (unsigned long long)v;
  const int pb = 63 - __clzll((long long)u);   // position of the leading bit
  const int be = pb + sc + 1023;               // biased exponent of the result
  if (be < 1 || be > 2045) return ldexp((double)v, sc);
  unsigned long long r;
  if (pb > 52) {
    const int sh = pb - 52;
    r = ((u >> (sh - 1)) + 1ull) >> 1;           // 53 bits, rounded; 2^53 on carry
  } else {
    r = u << (52 - pb);
  }
  // r in [2^52, 2^53]: adding it to (be - 1) << 52 sets the implicit bit's
  // exponent and carries a rounding overflow into the exponent.
  return __longlong_as_double((long long)(neg | ((((unsigned long long)(be - 1)) << 52) + r)));
}

// n / d for 0 <= n < 2^31 by an invariant multiplier (Granlund and Montgomery,
// PLDI 1994): with L = ceil(log2 d) and p = 31 + L, m = ceil(2^p / d) < 2^32
// and floor(n / d) = floor(n m / 2^p), because n m / 2^p exceeds n / d by
// less than n / 2^p < 2^-L <= 1 / d; d = 1 is the identity.
struct FastDiv {
  unsigned d, m;
  int sh;   // p - 32
};
inline FastDiv make_fastdiv(unsigned d) {
  FastDiv f{d, 0u, 0};
  if (d > 1) {
    int L = 0;
    while ((1ull << L) < d) ++L;
    const int p = 31 + L;
    f.m = (unsigned)(((1ull << p) + d - 1) / d);
    f.sh = p - 32;
  }
  return f;
}
__device__ __forceinline__ unsigned fdiv(unsigned n, const FastDiv& f) {
  return f.d == 1 ? n : (__umulhi(n, f.m) >> f.sh);
}

struct DerivArgs {
  const double2* src;   // nb arrays of G complex points (may equal dst)
  double2* dst;
  const uint4* op;      // operator digits, 2 S * TILE_B bytes in the canonical layout
  const int* ope;       // operator row exponents [NC]
  int nx, ny, nz;
  long long G;
  long long nlines;   // < 2^31
  int ntiles;
  FastDiv div1, div2;   // by nx, then by nz (lines along y) or ny (lines along z)
  FastDiv div0;         // by ny nz (lines along x: the array of a line)
  const double2* psi;   // kInResidual: psi (src is h psi); kOutUpdate: psi of the update
  const double* eps;    // kInResidual: eps per state (array b is state b / 2)
  const double* P;      // kOutScaleP: factor per point, times scale
  double scale;
  const float* w;       // kOutUpdate: weight per point, or null for 1
  int* status;
};

// First point and stride of line l (lines of one axis, x fastest, then the
// remaining axes in storage order, then the array).
template <int N, int AXIS>
__device__ __forceinline__ long long line_base(const DerivArgs& a, long long l, long long& stride) {
  if constexpr (AXIS == 0) {
    stride = 1;
    return l * N;
  } else {
    const unsigned lu = (unsigned)l;
    const unsigned t = fdiv(lu, a.div1), x = lu - t * (unsigned)a.nx;
    const unsigned b = fdiv(t, a.div2);
    if constexpr (AXIS == 1) {
      const unsigned z = t - b * (unsigned)a.nz;
      stride = a.nx;
      return (long long)b * a.G + (long long)(z * (unsigned)(a.ny * a.nx) + x);
    } else {
      const unsigned y = t - b * (unsigned)a.ny;
      stride = (long long)a.nx * a.ny;
      return (long long)b * a.G + (long long)(y * (unsigned)a.nx + x);
    }
  }
}

// Index b of the array that line l belongs to.
template <int N, int AXIS>
__device__ __forceinline__ unsigned line_array(const DerivArgs& a, long long l) {
  const unsigned lu = (unsigned)l;
  if constexpr (AXIS == 0) return fdiv(lu, a.div0);
  else return fdiv(fdiv(lu, a.div1), a.div2);
}

template <int N, int AXIS, int IN, int OUT>
__global__ void __launch_bounds__(THREADS, 1) k_oz_deriv(const DerivArgs a) {
  using Sh = Shape<N>;
  constexpr int NC = Sh::NC, STAGES = Sh::STAGES, HALF = Sh::HALF;
  constexpr int TILE_A = Sh::TILE_A, TILE_B = Sh::TILE_B, STAGE = Sh::STAGE;
  constexpr uint32_t TMEM_COLS = 512;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = (unsigned char*)(((unsigned long long)smem_raw + 1023ull) & ~1023ull);
  unsigned char* opb = base;                                  // operator digits
  unsigned char* ring = base + Sh::OPB;                       // STAGES x STAGE
  unsigned char* stg = ring + STAGES * STAGE;                 // [H0][producer thread] 16 B
  int* s_eb = (int*)(stg + Sh::STG);                          // [NC]
  int* s_ea = s_eb + NC;                                      // [2][BM]
  unsigned long long* bars = (unsigned long long*)(s_ea + 2 * BM);
  uint32_t* tmem_slot = (uint32_t*)(bars + kBars);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t bar0 = smem_u32(bars);
  auto full = [&](int s) { return bar0 + 8u * s; };
  auto empty = [&](int s) { return bar0 + 8u * (2 + s); };
  auto acc_full = [&](int b) { return bar0 + 8u * (4 + b); };
  auto acc_empty = [&](int b) { return bar0 + 8u * (4 + S + b); };
  auto ea_full = [&](int j) { return bar0 + 8u * (4 + 2 * S + j); };
  auto ea_empty = [&](int j) { return bar0 + 8u * (6 + 2 * S + j); };
  const uint32_t drain = bar0 + 8u * (8 + 2 * S);

  // the operator's digits and row exponents, for the whole launch
  for (int i = threadIdx.x; i < Sh::OPB / 16; i += blockDim.x) ((uint4*)opb)[i] = a.op[i];
  for (int i = threadIdx.x; i < NC; i += blockDim.x) s_eb[i] = a.ope[i];
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full(s), kProd * 32);
      mbar_init(empty(s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(acc_full(b), 1);
      mbar_init(acc_empty(b), kEpi);
    }
    for (int j = 0; j < 2; ++j) {
      mbar_init(ea_full(j), kProd * 32);
      mbar_init(ea_empty(j), kEpi * 32);
    }
    mbar_init(drain, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == kProd) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp < kProd) {
    // ---------------------------------------------------------------- producers
    // half 0 takes points [0, H0), half 1 [H0, N): H0 a multiple of 4, so each
    // half covers whole 16-byte chunks (8 reals) of the digit rows.  With
    // PREFETCH a thread copies its half line of the next tile into its own
    // staging slots (cp.async) while it splits the current one: no other
    // thread takes part in the hand-over.
    constexpr int H0 = Sh::H0, H1 = N - H0;
    static_assert(H1 > 0 && H1 <= H0 && H1 % 4 == 0, "line halves");
    constexpr int PT = kProd * 32;            // producer threads
    const int r = warp * 16 + (lane & 15);    // row (line) of the tile
    const int hh = lane >> 4;                 // which half of the line
    const int np = hh ? H1 : H0;              // points of this half
    const int p0 = hh ? H0 : 0;               // first point
    const uint32_t my_stg = smem_u32(stg) + (uint32_t)threadIdx.x * 16u;
    auto prefetch = [&](int t, bool go) {     // go: a data dependency on the caller's reads
      const long long l = (long long)t * BM + r;
      const bool valid = go && l < a.nlines;
      long long stride = 0;
      const long long lb = valid ? line_base<N, AXIS>(a, l, stride) : 0;
#pragma unroll
      for (int j = 0; j < H0; ++j)
        if (j < np)
          cp_async16(my_stg + (uint32_t)(j * PT * 16),
                     valid ? (const void*)(a.src + lb + (long long)(p0 + j) * stride)
                           : (const void*)a.src,
                     valid);
      cp_async_commit();
    };
    constexpr bool PF = Sh::PREFETCH && IN == kInPlain;
    if constexpr (PF)
      if (blockIdx.x < a.ntiles) prefetch(blockIdx.x, true);
    int it = 0;
    for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x, ++it) {
      const int s = it % STAGES, u = it / STAGES, slot = it & 1;
      double2 v[H0];
      if constexpr (PF) {
        cp_async_wait_all();
#pragma unroll
        for (int j = 0; j < H0; ++j)
          v[j] = j < np ? *(const double2*)(stg + (j * PT + threadIdx.x) * 16)
                        : make_double2(0.0, 0.0);
      } else {
        const long long l = (long long)t * BM + r;
        const bool valid = l < a.nlines;
        long long stride = 0;
        const long long lb = valid ? line_base<N, AXIS>(a, l, stride) : 0;
#pragma unroll
        for (int j = 0; j < H0; ++j)
          v[j] = (valid && j < np) ? a.src[lb + (long long)(p0 + j) * stride]
                                   : make_double2(0.0, 0.0);
        if constexpr (IN == kInResidual) {    // src - eps psi (src = h psi)
          const double e = valid ? a.eps[line_array<N, AXIS>(a, l) >> 1] : 0.0;
#pragma unroll
          for (int j = 0; j < H0; ++j)
            if (valid && j < np) {
              const double2 ps = a.psi[lb + (long long)(p0 + j) * stride];
              v[j] = make_double2(fma(-e, ps.x, v[j].x), fma(-e, ps.y, v[j].y));
            }
        }
      }
      int E = INT_MIN;
#pragma unroll
      for (int j = 0; j < H0; ++j) E = max(E, max(exp_of(v[j].x), exp_of(v[j].y)));
      if constexpr (PF) {
        // the next copy overwrites the slots just read: it is issued after E,
        // which depends on every value read
        if (t + (int)gridDim.x < a.ntiles) prefetch(t + gridDim.x, E != INT_MAX);
      }
      E = max(E, __shfl_xor_sync(0xffffffffu, E, 16));
      if (E == INT_MIN) E = 0;
      if (u > 0 && !mbar_wait(empty(s), (uint32_t)((u - 1) & 1))) {
        flag_status(a.status, SKY_ETIMEOUT);
        break;
      }
      if (it >= 2 && !mbar_wait(ea_empty(slot), (uint32_t)(((it >> 1) - 1) & 1))) {
        flag_status(a.status, SKY_ETIMEOUT);
        break;
      }
      if (hh == 0) s_ea[slot * BM + r] = E;
      unsigned char* ta = ring + s * STAGE;
#pragma unroll
      for (int c = 0; c < H0 / 4; ++c) {
        if (c < np / 4) {
          unsigned w[S][4];   // digit p of the chunk's 8 reals, as 4 bf16 pairs
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            float dr[S], di[S];
            digits6f(v[4 * c + j].x, E, dr);
            digits6f(v[4 * c + j].y, E, di);
#pragma unroll
            for (int p = 0; p < S; ++p) w[p][j] = bf16x2(dr[p], di[p]);
          }
          const int k0 = 2 * p0 + 8 * c;
#pragma unroll
          for (int p = 0; p < S; ++p)
            *(uint4*)(ta + p * TILE_A + cm_off(r, k0, NC)) =
                make_uint4(w[p][0], w[p][1], w[p][2], w[p][3]);
        }
      }
      // columns 2N .. NC - 1 (padding): zeros, from the second half
      if (hh == 1) {
#pragma unroll
        for (int k = 2 * N; k < NC; k += 8)
#pragma unroll
          for (int p = 0; p < S; ++p)
            *(uint4*)(ta + p * TILE_A + cm_off(r, k, NC)) = make_uint4(0u, 0u, 0u, 0u);
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_arrive(full(s));
      mbar_arrive(ea_full(slot));
    }
    if constexpr (PF) cp_async_wait_all();   // no copy outlives the launch
  } else if (warp == kProd) {
    // ---------------------------------------------------------------- MMA issue
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16(BM, NC);
      const uint32_t sb = smem_u32(opb);
      bool ok = true;
      int it = 0;
      for (int t = blockIdx.x; t < a.ntiles && ok; t += gridDim.x, ++it) {
        const int s = it % STAGES, u = it / STAGES;
        if (!mbar_wait(full(s), (uint32_t)(u & 1))) {
          flag_status(a.status, SKY_ETIMEOUT);
          break;
        }
        fence_after();
        const uint32_t sa = smem_u32(ring + s * STAGE);
        constexpr int NBUF = Sh::NBUF;
        const int b = it % NBUF, use = it / NBUF;
        if (use > 0) {
          // the epilogue must have drained this accumulator set
          if (!mbar_wait(acc_empty(b), (uint32_t)((use - 1) & 1))) {
            flag_status(a.status, SKY_ETIMEOUT);
            ok = false;
            break;
          }
          fence_after();
        }
        for (int g = 0; g <= S - 1; ++g) {
          // weights 0..3 into groups 0..3; weights 4 and 5 into group 4, the
          // weight-5 products with the operator's digits times 2^-8
          const int grp = g < NG ? g : NG - 1;
          const uint32_t acc = tmem + (uint32_t)(b * 256 + grp * NC);
          for (int p = 0; p <= g; ++p) {
            const int q = (g == S - 1) ? S + (g - p) : (g - p);
#pragma unroll
            for (int ks = 0; ks < NC / 16; ++ks)   // 16 values of K = two core matrices
              mma_bf16(acc, ns_desc(sa + p * TILE_A + ks * 256, NC),
                       ns_desc(sb + q * TILE_B + ks * 256, NC), idesc,
                       (g < NG && p == 0 && ks == 0) ? 0u : 1u);
          }
        }
        mma_commit(acc_full(b));   // arrives when this tile's MMAs have completed
        if (!ok) break;
        mma_commit(empty(s));
      }
      // every MMA issued by this thread completes before TMEM is freed
      mma_commit(drain);
      if (!mbar_wait(drain, 0)) flag_status(a.status, SKY_ETIMEOUT);
    }
  } else {
    // ---------------------------------------------------------------- epilogue
    const int w = warp - kProd - 1;            // 0 .. kEpi - 1
    const int q = warp & 3, half = w >> 2;     // TMEM lane quadrant = warp id mod 4
    const int row = q * 32 + lane;
    bool ok = true;
    int it = 0;
    for (int t = blockIdx.x; t < a.ntiles && ok; t += gridDim.x, ++it) {
      const int slot = it & 1;
      if (!mbar_wait(ea_full(slot), (uint32_t)((it >> 1) & 1))) {
        if (lane == 0) flag_status(a.status, SKY_ETIMEOUT);
        break;
      }
      const int E = s_ea[slot * BM + row];
      mbar_arrive(ea_empty(slot));
      const long long l = (long long)t * BM + row;
      long long stride = 0;
      const long long lb = l < a.nlines ? line_base<N, AXIS>(a, l, stride) : 0;
      long long bG = 0;
      if constexpr (OUT != kOutPlain) bG = l < a.nlines ? (long long)line_array<N, AXIS>(a, l) * a.G : 0;
      const int sc = E - 16 - 8 * (S - 1);
      constexpr int NBUF = Sh::NBUF;
      const int b = it % NBUF, use = it / NBUF;
      if (!mbar_wait(acc_full(b), (uint32_t)(use & 1))) {
        if (lane == 0) flag_status(a.status, SKY_ETIMEOUT);
        break;
      }
      fence_after();
      // columns in blocks of 8 (4 points).  The exact group sums (integers,
      // |G_g| < 2^24) fold into int32: u = G0 2^8 + G1, w = G2 2^8 + G3, and
      // x = round(2^8 G45) from the weight-{4,5} group (|x| < 2^31 for
      // K <= 64); the total sum_g G_g 2^{8(5-g)} = u 2^32 + w 2^16 + x.
#pragma unroll 1
      for (int cb = 0; cb < HALF; cb += 8) {
        uint32_t v[NG][8];
#pragma unroll
        for (int g = 0; g < NG; ++g)
          oz::tmem_ld<8>(tmem + ((uint32_t)(q * 32) << 16) +
                             (uint32_t)(b * 256 + g * NC + half * HALF + cb),
                         v[g]);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        long long acc[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          const int fu = __float2int_rn(__uint_as_float(v[0][c])) * 256 +
                         __float2int_rn(__uint_as_float(v[1][c]));
          const int fw = __float2int_rn(__uint_as_float(v[2][c])) * 256 +
                         __float2int_rn(__uint_as_float(v[3][c]));
          const int fx = __float2int_rn(__uint_as_float(v[4][c]) * 256.0f);
          acc[c] = ((long long)fu << 32) + ((long long)fw << 16) + (long long)fx;
        }
        if (l < a.nlines) {
#pragma unroll
          for (int c = 0; c < 8; c += 2) {
            const int o = half * HALF + cb + c;   // even: (re, im) of point o / 2
            const int m = o >> 1;
            if (m < N) {
              double2 res;
              res.x = scaled_double(acc[c], sc + s_eb[o]);
              res.y = scaled_double(acc[c + 1], sc + s_eb[o + 1]);
              const long long at = lb + m * stride;
              if constexpr (OUT == kOutScaleP) {
                const double f = a.P[at - bG] * a.scale;
                res = make_double2(res.x * f, res.y * f);
              } else if constexpr (OUT == kOutUpdate) {
                const double2 ps = a.psi[at];
                if (a.w) {
                  const double f = (double)a.w[at - bG];
                  res = make_double2(fma(-f, res.x, ps.x), fma(-f, res.y, ps.y));
                } else {
                  res = make_double2(ps.x - res.x, ps.y - res.y);
                }
              }
              a.dst[at] = res;
            }
          }
        }
      }
      // this warp's lanes of the accumulator set are read: hand it back
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(acc_empty(b));
    }
  }
  fence_before();
  __syncthreads();
  if (warp == kProd) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(TMEM_COLS)
                 : "memory");
  }
}

// ------------------------------------------------------------ host side
bool supported(int n) { return n == 8 || n == 12 || n == 16 || n == 20 || n == 24 || n == 32; }

// Digits [2S][NC][NC] (canonical layout, bf16 bit patterns; digits S..2S-1
// are digits 0..S-1 times 2^-8) and row exponents [NC] of the real operator
// of one axis, built in long double.  kind: kOpDeriv the derivative, the
// circulant D[m][q] = d[(m - q) mod n], d[r] = (i/n) sum_a kappa_a
// e^{2 pi i a r / n}; kOpFwd / kOpInv the unnormalised DFT, D[m][q] =
// e^{-+2 pi i (m q mod n) / n}.
void build_operator(int n, double L, double theta, int kind, std::vector<unsigned short>& dig,
                    std::vector<int>& ex) {
  const int NC = nc_of(n);
  const long double two_pi = 6.283185307179586476925286766559005768L;
  std::vector<long double> dre(n), dim(n);
  if (kind == kOpDeriv) {
    for (int r = 0; r < n; ++r) {
      long double sr = 0.0L, si = 0.0L;
      for (int a = 0; a < n; ++a) {
        const int mm = a < (n + 1) / 2 ? a : a - n;
        const long double kap = (two_pi * mm + (long double)theta) / (long double)L;
        const long double ang = two_pi * (long double)(((long long)a * r) % n) / (long double)n;
        sr -= kap * sinl(ang);   // Re of i kappa e^{i ang}
        si += kap * cosl(ang);   // Im
      }
      dre[r] = sr / n;
      dim[r] = si / n;
    }
  }
  auto entry = [&](int m, int q, double& re, double& im) {
    if (kind == kOpDeriv) {
      const int r = ((m - q) % n + n) % n;
      re = (double)dre[r];
      im = (double)dim[r];
    } else {
      const long double ang = two_pi * (long double)(((long long)m * q) % n) / (long double)n;
      re = (double)cosl(ang);
      im = (double)(kind == kOpFwd ? -sinl(ang) : sinl(ang));
    }
  };
  std::vector<double> B((size_t)NC * NC, 0.0);
  for (int m = 0; m < n; ++m)
    for (int q = 0; q < n; ++q) {
      double re, im;
      entry(m, q, re, im);
      B[(size_t)(2 * m) * NC + 2 * q] = re;
      B[(size_t)(2 * m) * NC + 2 * q + 1] = -im;
      B[(size_t)(2 * m + 1) * NC + 2 * q] = im;
      B[(size_t)(2 * m + 1) * NC + 2 * q + 1] = re;
    }
  dig.assign((size_t)2 * S * NC * NC, 0);
  ex.assign(NC, 0);
  for (int o = 0; o < NC; ++o) {
    int F = INT_MIN;
    for (int k = 0; k < NC; ++k) {
      const double x = B[(size_t)o * NC + k];
      if (x != 0.0) {
        int e;
        std::frexp(x, &e);   // |x| < 2^e
        F = e > F ? e : F;
      }
    }
    if (F == INT_MIN) F = 0;
    ex[o] = F;
    for (int k = 0; k < NC; ++k) {
      const double x = B[(size_t)o * NC + k];
      // X = round(|x| 2^{8S - F}) < 2^48 + 1, exact (power-of-two scaling, then +0.5)
      long long X = (long long)std::floor(std::ldexp(std::fabs(x), 8 * S - F) + 0.5);
      int d[S];
      for (int s = S - 1; s >= 1; --s) {
        int v = (int)(X & 255);
        X >>= 8;
        if (v >= 128) { v -= 256; ++X; }
        d[s] = v;
      }
      d[0] = (int)X;
      for (int p = 0; p < S; ++p) {
        const float f = (float)(x < 0.0 ? -d[p] : d[p]);   // |d| <= 256: exact in bf16
        const float f8 = f * 0.00390625f;                   // times 2^-8: also exact
        unsigned u, u8;
        std::memcpy(&u, &f, 4);
        std::memcpy(&u8, &f8, 4);
        dig[((size_t)p * NC * NC * 2 + cm_off(o, k, NC)) / 2] = (unsigned short)(u >> 16);
        dig[((size_t)(S + p) * NC * NC * 2 + cm_off(o, k, NC)) / 2] = (unsigned short)(u8 >> 16);
      }
    }
  }
}

template <int N, int AXIS, int IN, int OUT>
cudaError_t launch(const DerivArgs& a, const Ctx* c) {
  using Sh = Shape<N>;
  static bool set[64] = {false};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (!set[dev]) {
    e = cudaFuncSetAttribute(k_oz_deriv<N, AXIS, IN, OUT>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, Sh::SMEM);
    if (e != cudaSuccess) return e;
    set[dev] = true;
  }
  const int grid = a.ntiles < c->num_sms ? a.ntiles : c->num_sms;
  k_oz_deriv<N, AXIS, IN, OUT><<<grid, THREADS, Sh::SMEM, c->stream>>>(a);
  note_launch();
  return cudaGetLastError();
}

}  // namespace ozd

static sky_status upload_operator(Ctx* c, int n, double L, double theta, int kind, void** dig_out,
                                  int** ex_out) {
  std::vector<unsigned short> dig;
  std::vector<int> ex;
  ozd::build_operator(n, L, theta, kind, dig, ex);
  cudaError_t e = cudaMalloc(dig_out, dig.size() * sizeof(unsigned short));
  if (e == cudaSuccess) e = cudaMalloc(ex_out, ex.size() * sizeof(int));
  if (e == cudaSuccess)
    e = cudaMemcpy(*dig_out, dig.data(), dig.size() * sizeof(unsigned short), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(*ex_out, ex.data(), ex.size() * sizeof(int), cudaMemcpyHostToDevice);
  return cuda_check(c, e, "operator upload");
}

sky_status deriv_tc_init(Ctx* c) {
  for (int j = 0; j < 3; ++j) {
    c->d_dop[j] = nullptr;
    c->d_dope[j] = nullptr;
    for (int k = 0; k < 2; ++k) {
      c->d_dft[j][k] = nullptr;
      c->d_dfte[j][k] = nullptr;
    }
  }
  if (c->prec != SKY_F64) return SKY_OK;
  for (int j = 0; j < 3; ++j) {
    if (!ozd::supported(c->n[j])) continue;
    sky_status s = upload_operator(c, c->n[j], c->L[j], c->theta[j], ozd::kOpDeriv, &c->d_dop[j],
                                   &c->d_dope[j]);
    for (int k = 0; k < 2 && s == SKY_OK; ++k)
      s = upload_operator(c, c->n[j], c->L[j], c->theta[j], k == 0 ? ozd::kOpFwd : ozd::kOpInv,
                          &c->d_dft[j][k], &c->d_dfte[j][k]);
    if (s != SKY_OK) return s;
  }
  return SKY_OK;
}

namespace {

ozd::DerivArgs op_args(const Ctx* c, int ax, const double2* src, double2* dst, long long nb,
                       const void* op, const int* ope) {
  ozd::DerivArgs a{};
  a.src = src;
  a.dst = dst;
  a.op = (const uint4*)op;
  a.ope = ope;
  a.nx = c->n[0];
  a.ny = c->n[1];
  a.nz = c->n[2];
  a.G = c->G;
  a.nlines = nb * (c->G / c->n[ax]);
  a.div1 = ozd::make_fastdiv((unsigned)c->n[0]);
  a.div2 = ozd::make_fastdiv((unsigned)(ax == 1 ? c->n[2] : c->n[1]));
  a.div0 = ozd::make_fastdiv((unsigned)(c->n[1] * c->n[2]));
  const long long nt = (a.nlines + ozd::BM - 1) / ozd::BM;
  a.ntiles = nt > INT_MAX ? INT_MAX : (int)nt;
  a.status = c->d_status;
  return a;
}

// One operator pass along ax with the given modes (only the combinations
// the library uses are instantiated).
template <int IN, int OUT>
cudaError_t op_pass(const Ctx* c, int ax, const ozd::DerivArgs& a) {
  if (a.nlines == 0) return cudaSuccess;
  if (a.nlines >= (1LL << 31)) return cudaErrorInvalidValue;
  auto go = [&](auto NC) -> cudaError_t {
    constexpr int N = decltype(NC)::value;
    if constexpr (IN == ozd::kInResidual) {
      return ax == 2 ? ozd::launch<N, 2, IN, OUT>(a, c) : cudaErrorInvalidValue;
    } else if constexpr (OUT == ozd::kOutScaleP) {
      return ax == 0 ? ozd::launch<N, 0, IN, OUT>(a, c) : cudaErrorInvalidValue;
    } else if constexpr (OUT == ozd::kOutUpdate) {
      return ax == 2 ? ozd::launch<N, 2, IN, OUT>(a, c) : cudaErrorInvalidValue;
    } else {
      if (ax == 0) return ozd::launch<N, 0, IN, OUT>(a, c);
      if (ax == 1) return ozd::launch<N, 1, IN, OUT>(a, c);
      return ozd::launch<N, 2, IN, OUT>(a, c);
    }
  };
  switch (c->n[ax]) {
    case 8: return go(std::integral_constant<int, 8>{});
    case 12: return go(std::integral_constant<int, 12>{});
    case 16: return go(std::integral_constant<int, 16>{});
    case 20: return go(std::integral_constant<int, 20>{});
    case 24: return go(std::integral_constant<int, 24>{});
    case 32: return go(std::integral_constant<int, 32>{});
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

// dst = d_ax src over nb arrays of G complex doubles (dst may equal src).
cudaError_t deriv_tc(Ctx* c, int ax, const double2* src, double2* dst, long long nb) {
  if (!c->d_dop[ax]) return cudaErrorInvalidValue;
  return op_pass<ozd::kInPlain, ozd::kOutPlain>(
      c, ax, op_args(c, ax, src, dst, nb, c->d_dop[ax], c->d_dope[ax]));
}

bool damp_tc_available(const Ctx* c) {
  for (int j = 0; j < 3; ++j)
    if (!c->d_dft[j][0] || !c->d_dft[j][1]) return false;
  return true;
}

// The damped step's 3D transform pair as six operator passes over the 2I
// arrays (the damping table P must be current): phi = F_z F_y F_x of
// (h psi - eps psi), times P x0 / G in the last forward pass, the inverse
// passes, phi = psi - w (result) in the last.
cudaError_t damp_tc(Ctx* c, int q, const double2* psi, const double2* hpsi, const double* eps,
                    double2* phi, int I, double x0, const float* w) {
  const long long nb = 2LL * I;
  auto args = [&](int ax, int k, const double2* src) {
    return op_args(c, ax, src, phi, nb, c->d_dft[ax][k], c->d_dfte[ax][k]);
  };
  ozd::DerivArgs a = args(2, 0, hpsi);
  a.psi = psi;
  a.eps = eps;
  cudaError_t e = op_pass<ozd::kInResidual, ozd::kOutPlain>(c, 2, a);
  if (e == cudaSuccess) e = op_pass<ozd::kInPlain, ozd::kOutPlain>(c, 1, args(1, 0, phi));
  if (e == cudaSuccess) {
    ozd::DerivArgs b = args(0, 0, phi);
    b.P = c->d_damp[q];
    b.scale = x0 / (double)c->G;
    e = op_pass<ozd::kInPlain, ozd::kOutScaleP>(c, 0, b);
  }
  if (e == cudaSuccess) e = op_pass<ozd::kInPlain, ozd::kOutPlain>(c, 0, args(0, 1, phi));
  if (e == cudaSuccess) e = op_pass<ozd::kInPlain, ozd::kOutPlain>(c, 1, args(1, 1, phi));
  if (e == cudaSuccess) {
    ozd::DerivArgs d = args(2, 1, phi);
    d.psi = psi;
    d.w = w;
    e = op_pass<ozd::kInPlain, ozd::kOutUpdate>(c, 2, d);
  }
  return e;
}

}  // namespace sky
