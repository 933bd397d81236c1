// Exact-integer split GEMM on the 5th-generation tensor cores (sm_103a) for the
// FP64 and FP32 forms of the overlap / Hamiltonian matrices (Eqs. normmatrix,
// hammatrix) and of the recombination (Sec. 3.3.3).
//
// Each row r of an operand is scaled by a power of two 2^e[r] (|x| < 2^e[r])
// and written as S signed base-256 digits,
//     x = 2^e[r] sum_{s<S} alpha_s 2^{-8(s+1)}   (+ a remainder below 2^{-8S}),
// |alpha_0| <= 256, |alpha_s| <= 128 (s >= 1): small integers that bf16
// holds exactly ("slices", Ozaki, Ogita, Oishi and Rump 2012).  The product
// keeps the slice pairs of total weight g = s + t <= S - 1:
//     sum_k A[m][k] B[n][k] = 2^{e_m + f_n - 16} sum_g 2^{-8g} G_g[m][n],
//     G_g = sum_{s + t = g} alpha_s beta_t^T.
// Every G_g is a sum of integer products, so its FP32 accumulation in TMEM is
// exact as long as it stays below 2^24: per K value |G_g| <= (g + 3) 2^14
// (g >= 1) or 2^16 (g = 0), so a segment of 128 values of K (4 K blocks of
// 32) is exact for every g <= 5.  One TMEM accumulator per group; group g is
// drained ("flushed") after each of its segments, and the segments of
// different groups end at different K blocks (staggered by g mod 4), so the
// MMA warp waits only for the one group being drained.  The drained exact
// sums are added, scaled by 2^{-8g}, into an unevaluated FP32 pair (hi, lo)
// per output element by error-free TwoSum (about 48 significant bits).
//
// Persistent kernel, one CTA per SM; work items are (128 x BNT output tile,
// K range).  Warp roles:
//   warp 0     TMA producer: 3D cp.async.bulk.tensor loads of one 32-wide K
//              block of every slice of A (128 rows) and B (BNT rows), 64-byte
//              swizzle, into a ring of stages;
//   warp 1     owns TMEM (S accumulators of BNT fp32 columns) and one elected
//              lane issues tcgen05.mma (M = 128, N = BNT, K = 16): for each K
//              block and group g all products (s, g - s);
//   warps 2-9  epilogue: two warps per TMEM lane quadrant, each half of the
//              columns; drain a group when its segment ends, accumulate
//              (hi, lo); write the item's result at its end.
// Every mbarrier wait is bounded; a timeout sets SKY_ETIMEOUT in the status
// word, the kernel waits (bounded) for the MMAs it issued, frees TMEM and
// returns.
#pragma once

#include "tc_gemm.cuh"

namespace sky {
namespace oz {

using tc::fence_after;
using tc::fence_before;
using tc::idesc_bf16;
using tc::mbar_expect_tx;
using tc::mbar_init;
using tc::mbar_wait;
using tc::mma_bf16;
using tc::mma_commit;
using tc::smem_u32;

constexpr int BM = 128;
constexpr int BK = 32;                    // bf16 K block: one 64-byte swizzle row
constexpr int kSegKB = 4;                 // K blocks per exact segment (128 values)
constexpr int kEpiWarps = 8;
constexpr int THREADS = 64 + 32 * kEpiWarps;
constexpr int kMaxS = 6;
constexpr int kMaxStages = 4;
constexpr int kSmemMax = 232448;          // dynamic shared memory opt-in limit per CTA
constexpr int kSmemExtra = 1024 + 256;    // alignment slack + barriers
constexpr int TILE_A = BM * BK * 2;       // 8 KiB per A slice tile

// Slices of the FP64 and FP32 forms and their tile widths (S groups x BNT
// columns of TMEM <= 512).
constexpr int kS64 = 6, kBN64 = 80;
constexpr int kS32 = 4, kBN32 = 96;

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int c0, int c1,
                                            int c2, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
      "l"((unsigned long long)map), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
      : "memory");
}
// Shared-memory matrix descriptor: K-major tile with 64-byte swizzle, rows of
// 64 bytes, 8-row groups 512 bytes apart (stride byte offset), descriptor
// version 1, layout type 4 (64B swizzle).
__device__ __forceinline__ uint64_t sw64_desc(uint32_t saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | (1ull << 16) | (32ull << 32) | (1ull << 46) |
         (4ull << 61);
}
// NC consecutive fp32 columns (NC = 8, 16 or 32) of this warp's 32 TMEM lanes.
template <int NC>
__device__ __forceinline__ void tmem_ld(uint32_t taddr, uint32_t* r);
template <>
__device__ __forceinline__ void tmem_ld<8>(uint32_t taddr, uint32_t* r) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                 "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
}
template <>
__device__ __forceinline__ void tmem_ld<16>(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
      "%12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
template <>
__device__ __forceinline__ void tmem_ld<32>(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, "
      "%28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
        "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
        "=r"(r[31])
      : "r"(taddr));
}
// Columns [0, NC) of a warp's share, NC = 40 or 48, as 32 + 8 or 32 + 16.
template <int NC>
__device__ __forceinline__ void tmem_ld_cols(uint32_t taddr, uint32_t* r) {
  static_assert(NC == 40 || NC == 48, "column share");
  tmem_ld<32>(taddr, r);
  tmem_ld<NC - 32>(taddr + 32, r + 32);
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Group g's segment ends after K block j (of nkb in the item): every kSegKB
// blocks, offset by g mod kSegKB, and at the item's last block.
__device__ __forceinline__ bool flush_at(int j, int g, int nkb) {
  return j == nkb - 1 || ((j + 1 + (g % kSegKB)) % kSegKB) == 0;
}

struct OzArgs {
  int M, N, K;              // rows of A, rows of B, K (bf16 elements, within the maps)
  int kb_per_split;         // K blocks per split
  int nsplit;               // K splits
  int tri;                  // overlap lower-triangle pruning: B = [b; b'] with I rows each
  int I;
  int ntiles;               // output tiles in use (pruned when tri)
  int mode;                 // 0: (hi, lo) partials; 1: scaled final output
  float2* P;                // mode 0: P[z][m][n], row stride ldp, split stride sp
  long long ldp, sp;
  void* out;                // mode 1: out[m][n] (double, or float when out_f32), row stride ldo
  long long ldo;
  int out_f32;
  const int* ea;            // mode 1: row exponents of A [M]
  const int* eb;            // mode 1: row exponents of B, eb[n >> eb_shift]
  int eb_shift;
  int* status;
  const int* run;           // device gate: the launch does nothing when *run == 0 or *stop != 0
  const int* stop;
};

// First 128-row tile a column tile of the [b; b'] overlap layout needs
// (rows a >= the smallest state index b its columns hold).
__host__ __device__ inline int tri_mi_min(int nj, int bnt, int N, int I) {
  const int n0 = nj * bnt;
  int n1 = n0 + bnt;
  if (n1 > N) n1 = N;
  --n1;
  const int bmin = (n0 < I && n1 >= I) ? 0 : (n0 < I ? n0 : n0 - I);
  return bmin / BM;
}

__host__ __device__ inline void item_of(const OzArgs& a, int bnt, int t, int& m0, int& n0, int& kb0,
                                        int& nkb) {
  const int mt = (a.M + BM - 1) / BM, nt = (a.N + bnt - 1) / bnt;
  const int z = t / a.ntiles;
  int tt = t - z * a.ntiles;
  int mi, nj;
  if (!a.tri) {
    mi = tt % mt;
    nj = tt / mt;
  } else {
    nj = 0;
    for (; nj < nt; ++nj) {
      int lo = tri_mi_min(nj, bnt, a.N, a.I);
      if (lo > mt) lo = mt;
      const int cnt = mt - lo;
      if (tt < cnt) break;
      tt -= cnt;
    }
    int lo = tri_mi_min(nj, bnt, a.N, a.I);
    if (lo > mt) lo = mt;
    mi = lo + tt;
  }
  m0 = mi * BM;
  n0 = nj * bnt;
  const int nkb_total = (a.K + BK - 1) / BK;
  kb0 = z * a.kb_per_split;
  nkb = nkb_total - kb0;
  if (nkb > a.kb_per_split) nkb = a.kb_per_split;
  if (nkb < 0) nkb = 0;
}

// Grouped products: np independent n x n complex products in one launch
// (the many small problems of a batched eigensolve).  Problem b's operand
// rows are stacked in the two maps (A rows ra[b] .. ra[b] + n - 1, B rows
// rb[b] .. rb[b] + 2n - 1, K = 2n digits per row, zero beyond); its items
// are the output tiles tile0[b] .. tile0[b+1] - 1 (one K range each); its
// partials go to P + po[b], rows of 2n.  A tile that runs past the problem's
// rows reads the next problem's rows, whose results are not stored.
struct OzGroup {
  int np;
  int tile0[kMaxBatch + 1];
  int n[kMaxBatch];
  int ra[kMaxBatch];
  int rb[kMaxBatch];
  long long po[kMaxBatch];
  const double2* A[kMaxBatch];
  const double2* B[kMaxBatch];
  double2* C[kMaxBatch];
  const int* run[kMaxBatch];
  const int* stop[kMaxBatch];
};

__host__ __device__ inline bool group_gated(const OzGroup& G, int b) {
  return (G.run[b] && *G.run[b] == 0) || (G.stop[b] && *G.stop[b] != 0);
}

// One work item: global map rows m0 (A) and n0 (B), K blocks kb0 .. kb0 +
// nkb - 1, output rows / columns from (mloc, nloc) within an M x N result
// (of problem b in a grouped launch).
struct OzItem {
  int m0, n0, kb0, nkb, b, mloc, nloc, M, N;
};

template <bool GROUP>
__device__ __forceinline__ bool item_at(const OzArgs& a, const OzGroup* G, int bnt, int t,
                                        OzItem& it) {
  if constexpr (GROUP) {
    int lo = 0, hi = G->np - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (G->tile0[mid] <= t) lo = mid; else hi = mid - 1;
    }
    const int b = lo, n = G->n[b];
    if (group_gated(*G, b)) return false;
    const int mt = (n + BM - 1) / BM, tt = t - G->tile0[b];
    const int mi = tt % mt, nj = tt / mt;
    it.b = b;
    it.mloc = mi * BM;
    it.nloc = nj * bnt;
    it.m0 = G->ra[b] + it.mloc;
    it.n0 = G->rb[b] + it.nloc;
    it.kb0 = 0;
    it.nkb = (2 * n + BK - 1) / BK;
    it.M = n;
    it.N = 2 * n;
  } else {
    item_of(a, bnt, t, it.m0, it.n0, it.kb0, it.nkb);
    it.b = t / a.ntiles;   // the K split
    it.mloc = it.m0;
    it.nloc = it.n0;
    it.M = a.M;
    it.N = a.N;
  }
  return true;
}

__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float y) {
  const float s = hi + y;
  const float bp = s - hi;
  const float e = (hi - (s - bp)) + (y - bp);
  hi = s;
  lo += e;
}

// 2^k as a double (k in the normal range).
__device__ __forceinline__ double pow2d(int k) {
  return __longlong_as_double((long long)(1023 + k) << 52);
}

template <int S, int BNT, bool GROUP>
__device__ __forceinline__ void oz_gemm_body(const CUtensorMap* pA, const CUtensorMap* pB,
                                             const OzArgs& a, const OzGroup* grp) {
  if ((a.run && *a.run == 0) || (a.stop && *a.stop != 0)) return;   // uniform in the CTA
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = (unsigned char*)(((unsigned long long)smem_raw + 1023ull) & ~1023ull);
  constexpr int TILE_B = BNT * BK * 2;
  constexpr int STAGE = S * (TILE_A + TILE_B);
  constexpr int STAGES = (kSmemMax - kSmemExtra) / STAGE < kMaxStages
                             ? (kSmemMax - kSmemExtra) / STAGE
                             : kMaxStages;
  static_assert(STAGES >= 2, "ring");
  static_assert(S * BNT <= 512, "TMEM");
  static_assert(TILE_B % 1024 == 0, "swizzle alignment");
  constexpr uint32_t TMEM_COLS = 512;
  constexpr int HALF = BNT / 2;
  unsigned long long* bars = (unsigned long long*)(base + STAGES * STAGE);
  uint32_t* tmem_slot = (uint32_t*)(bars + 2 * kMaxStages + 2 * kMaxS + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nitems = GROUP ? grp->tile0[grp->np] : a.ntiles * a.nsplit;
  const uint32_t bar0 = smem_u32(bars);
  auto full = [&](int s) { return bar0 + 8u * s; };
  auto empty = [&](int s) { return bar0 + 8u * (kMaxStages + s); };
  auto acc_full = [&](int g) { return bar0 + 8u * (2 * kMaxStages + g); };
  auto acc_empty = [&](int g) { return bar0 + 8u * (2 * kMaxStages + kMaxS + g); };
  const uint32_t drain = bar0 + 8u * (2 * kMaxStages + 2 * kMaxS);

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full(s), 1);
      mbar_init(empty(s), 1);
    }
    for (int g = 0; g < S; ++g) {
      mbar_init(acc_full(g), 1);
      mbar_init(acc_empty(g), kEpiWarps);   // one arrival per epilogue warp
    }
    mbar_init(drain, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
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

  if (warp == 0) {
    if (lane == 0) {
      // stage layout: A slices 0..S-1, then B slices 0..S-1
      long long g = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < nitems && ok; t += gridDim.x) {
        OzItem it;
        if (!item_at<GROUP>(a, grp, BNT, t, it)) continue;
        const int m0 = it.m0, n0 = it.n0, kb0 = it.kb0, nkb = it.nkb;
        for (int j = 0; j < nkb; ++j, ++g) {
          const int s = (int)(g % STAGES);
          const long long u = g / STAGES;
          if (u > 0 && !mbar_wait(empty(s), (uint32_t)((u - 1) & 1))) {
            flag_status(a.status, SKY_ETIMEOUT);
            ok = false;
            break;
          }
          const uint32_t sa = smem_u32(base + s * STAGE);
          mbar_expect_tx(full(s), STAGE);
          const int kc = (kb0 + j) * BK;
          for (int p = 0; p < S; ++p) {
            tma_load_3d(sa + p * TILE_A, pA, kc, m0, p, full(s));
            tma_load_3d(sa + S * TILE_A + p * TILE_B, pB, kc, n0, p, full(s));
          }
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16(BM, BNT);
      uint32_t nfl[S];
#pragma unroll
      for (int g = 0; g < S; ++g) nfl[g] = 0;
      long long gpos = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < nitems && ok; t += gridDim.x) {
        OzItem it;
        if (!item_at<GROUP>(a, grp, BNT, t, it)) continue;
        const int nkb = it.nkb;
        for (int j = 0; j < nkb && ok; ++j, ++gpos) {
          const int s = (int)(gpos % STAGES);
          const long long u = gpos / STAGES;
          if (!mbar_wait(full(s), (uint32_t)(u & 1))) {
            flag_status(a.status, SKY_ETIMEOUT);
            ok = false;
            break;
          }
          fence_after();
          const uint32_t sa = smem_u32(base + s * STAGE);
#pragma unroll
          for (int g = 0; g < S; ++g) {
            const bool seg_start = (j == 0) || flush_at(j - 1, g, nkb);
            if (seg_start && nfl[g] > 0) {
              // the epilogue must have drained this group's previous segment
              if (!mbar_wait(acc_empty(g), (nfl[g] - 1) & 1)) {
                flag_status(a.status, SKY_ETIMEOUT);
                ok = false;
                break;
              }
              fence_after();
            }
            const uint32_t acc = tmem + (uint32_t)(g * BNT);
#pragma unroll
            for (int p = 0; p <= g; ++p) {
              const uint64_t da = sw64_desc(sa + p * TILE_A);
              const uint64_t db = sw64_desc(sa + S * TILE_A + (g - p) * TILE_B);
#pragma unroll
              for (int k = 0; k < BK / 16; ++k)   // +32 bytes along K = +2 in the encoded address
                mma_bf16(acc, da + 2ull * k, db + 2ull * k, idesc,
                         (seg_start && p == 0 && k == 0) ? 0u : 1u);
            }
          }
          if (!ok) break;
          mma_commit(empty(s));
#pragma unroll
          for (int g = 0; g < S; ++g)
            if (flush_at(j, g, nkb)) {
              mma_commit(acc_full(g));   // arrives when this group's MMAs have completed
              ++nfl[g];
            }
        }
      }
      // every MMA issued by this thread completes before TMEM is freed
      mma_commit(drain);
      if (!mbar_wait(drain, 0)) flag_status(a.status, SKY_ETIMEOUT);
    }
  } else {
    // epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31, columns half * HALF ..
    const int q = warp & 3, half = (warp - 2) >> 2;
    uint32_t efl[S];
#pragma unroll
    for (int g = 0; g < S; ++g) efl[g] = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < nitems && ok; t += gridDim.x) {
      OzItem it;
      if (!item_at<GROUP>(a, grp, BNT, t, it)) continue;
      const int nkb = it.nkb;
      float hi[HALF], lo[HALF];
#pragma unroll
      for (int c = 0; c < HALF; ++c) hi[c] = lo[c] = 0.0f;
      for (int j = 0; j < nkb && ok; ++j) {
#pragma unroll
        for (int g = 0; g < S; ++g) {
          if (!flush_at(j, g, nkb)) continue;
          if (!mbar_wait(acc_full(g), efl[g] & 1)) {
            if (lane == 0) flag_status(a.status, SKY_ETIMEOUT);
            ok = false;
            break;
          }
          fence_after();
          uint32_t v[HALF];
          tmem_ld_cols<HALF>(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(g * BNT + half * HALF),
                             v);
          // this warp's lanes of the accumulator are read: hand it back
          fence_before();
          __syncwarp();
          if (lane == 0)
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(acc_empty(g)) : "memory");
          ++efl[g];
          const float sc = __int_as_float((127 - 8 * g) << 23);   // 2^{-8g}, exact
#pragma unroll
          for (int c = 0; c < HALF; ++c) two_sum_acc(hi[c], lo[c], __uint_as_float(v[c]) * sc);
        }
      }
      if (!ok) break;
      const int row = it.mloc + q * 32 + lane;
      const int col0 = it.nloc + half * HALF;
      if (row < it.M) {
        if (GROUP || a.mode == 0) {
          float2* prow = GROUP ? a.P + grp->po[it.b] + (long long)row * it.N
                               : a.P + (long long)it.b * a.sp + (long long)row * a.ldp;
#pragma unroll
          for (int c = 0; c < HALF; ++c)
            if (col0 + c < it.N) prow[col0 + c] = make_float2(hi[c], lo[c]);
        } else {
          const int er = a.ea[row] - 16;
          if (a.out_f32) {
            float* orow = (float*)a.out + (long long)row * a.ldo;
#pragma unroll
            for (int c = 0; c < HALF; ++c)
              if (col0 + c < a.N) {
                const double sc = pow2d(er + a.eb[(col0 + c) >> a.eb_shift]);
                orow[col0 + c] = (float)(((double)hi[c] + (double)lo[c]) * sc);
              }
          } else {
            double* orow = (double*)a.out + (long long)row * a.ldo;
#pragma unroll
            for (int c = 0; c < HALF; ++c)
              if (col0 + c < a.N) {
                const double sc = pow2d(er + a.eb[(col0 + c) >> a.eb_shift]);
                orow[col0 + c] = ((double)hi[c] + (double)lo[c]) * sc;
              }
          }
        }
      }
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 1) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(TMEM_COLS)
                 : "memory");
  }
}

template <int S, int BNT>
__global__ void __launch_bounds__(THREADS, 1)
    k_oz_gemm(const __grid_constant__ CUtensorMap mA, const __grid_constant__ CUtensorMap mB,
              OzArgs a) {
  oz_gemm_body<S, BNT, false>(&mA, &mB, a, nullptr);
}

template <int S, int BNT>
__global__ void __launch_bounds__(THREADS, 1)
    k_oz_gemm_group(const __grid_constant__ CUtensorMap mA, const __grid_constant__ CUtensorMap mB,
                    OzArgs a, const __grid_constant__ OzGroup grp) {
  oz_gemm_body<S, BNT, true>(&mA, &mB, a, &grp);
}

template <int S, int BNT>
constexpr int smem_bytes() {
  constexpr int stage = S * (TILE_A + BNT * BK * 2);
  constexpr int st = (kSmemMax - kSmemExtra) / stage < kMaxStages ? (kSmemMax - kSmemExtra) / stage
                                                                    : kMaxStages;
  return st * stage + kSmemExtra;
}

// 3D bf16 map: slices [S][rows][ld] (ld, slice stride in elements, multiples
// of 8), box BK x box_rows x 1, 64-byte swizzle; rows beyond `rows` and K
// beyond `K` read as zeros.
inline cudaError_t make_map3(CUtensorMap* map, const void* ptr, int S, int rows, int K, long long ld,
                             long long slice_stride, int box_rows) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                     cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
    encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
  }
  const cuuint64_t gdim[3] = {(cuuint64_t)K, (cuuint64_t)rows, (cuuint64_t)S};
  const cuuint64_t gstride[2] = {(cuuint64_t)ld * 2, (cuuint64_t)slice_stride * 2};
  const cuuint32_t box[3] = {(cuuint32_t)BK, (cuuint32_t)box_rows, 1};
  const cuuint32_t estride[3] = {1, 1, 1};
  CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(ptr), gdim,
                      gstride, box, estride, CU_TENSOR_MAP_INTERLEAVE_NONE,
                      CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// Number of output tiles of an M x N product (pruned to the tiles that hold
// an element a >= b of the [b; b'] overlap layout when tri).
inline int count_tiles(int M, int N, int bnt, bool tri, int I) {
  const int mt = (M + BM - 1) / BM, nt = (N + bnt - 1) / bnt;
  if (!tri) return mt * nt;
  int n = 0;
  for (int nj = 0; nj < nt; ++nj) {
    int lo = tri_mi_min(nj, bnt, N, I);
    if (lo > mt) lo = mt;
    n += mt - lo;
  }
  return n;
}

// Launch k_oz_gemm<S, BNT>.  A: slices [S][M][K] (row stride lda, slice
// stride sa), B: [S][N][K] (ldb, sb), all 16-byte aligned.  *splits in: the
// K splits wanted; out: the splits used (mode 0 writes P[z] for z < *splits).
template <int S, int BNT>
inline cudaError_t oz_gemm(const void* A, long long lda, long long sa, int M, const void* B,
                           long long ldb, long long sb, int N, int K, bool tri, int I, OzArgs g,
                           int* splits, cudaStream_t s) {
  if (M <= 0 || N <= 0 || K <= 0) { *splits = 0; return cudaSuccess; }
  if ((lda & 7) || (ldb & 7) || (sa & 7) || (sb & 7) || lda < K || ldb < K)
    return cudaErrorInvalidValue;
  CUtensorMap ma, mb;
  cudaError_t e;
  if ((e = make_map3(&ma, A, S, M, K, lda, sa, BM)) != cudaSuccess) return e;
  if ((e = make_map3(&mb, B, S, N, K, ldb, sb, BNT)) != cudaSuccess) return e;
  static bool smem_set[64] = {false};
  int dev = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (!smem_set[dev]) {
    e = cudaFuncSetAttribute(k_oz_gemm<S, BNT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             smem_bytes<S, BNT>());
    if (e != cudaSuccess) return e;
    smem_set[dev] = true;
  }
  const int nkb = (K + BK - 1) / BK;
  int z = *splits < 1 ? 1 : *splits;
  if (z > nkb) z = nkb;
  g.M = M; g.N = N; g.K = K;
  g.kb_per_split = (nkb + z - 1) / z;
  z = (nkb + g.kb_per_split - 1) / g.kb_per_split;
  g.nsplit = z;
  g.tri = tri ? 1 : 0;
  g.I = I;
  g.ntiles = count_tiles(M, N, BNT, tri, I);
  const long long items = (long long)g.ntiles * z;
  int nsm = 0;
  if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  const int grid = (int)(items < nsm ? items : nsm);
  k_oz_gemm<S, BNT><<<grid, THREADS, smem_bytes<S, BNT>(), s>>>(ma, mb, g);
  note_launch();
  *splits = z;
  return cudaGetLastError();
}

// Launch the grouped form over grp's problems: A holds rowsA stacked rows,
// B rowsB, both of row stride ld (bf16 elements, a multiple of 8; each
// problem's digits zero from K = 2n on), slice strides sa, sb.
template <int S, int BNT>
inline cudaError_t oz_gemm_group(const void* A, long long sa, int rowsA, const void* B,
                                 long long sb, int rowsB, long long ld, const OzGroup& grp,
                                 OzArgs g, cudaStream_t s) {
  if (grp.np <= 0 || grp.tile0[grp.np] == 0) return cudaSuccess;
  if ((ld & 7) || (sa & 7) || (sb & 7) || rowsA <= 0 || rowsB <= 0) return cudaErrorInvalidValue;
  CUtensorMap ma, mb;
  cudaError_t e;
  if ((e = make_map3(&ma, A, S, rowsA, (int)ld, ld, sa, BM)) != cudaSuccess) return e;
  if ((e = make_map3(&mb, B, S, rowsB, (int)ld, ld, sb, BNT)) != cudaSuccess) return e;
  static bool smem_set[64] = {false};
  int dev = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (!smem_set[dev]) {
    e = cudaFuncSetAttribute(k_oz_gemm_group<S, BNT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             smem_bytes<S, BNT>());
    if (e != cudaSuccess) return e;
    smem_set[dev] = true;
  }
  int nsm = 0;
  if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  const int items = grp.tile0[grp.np];
  const int grid = items < nsm ? items : nsm;
  g.mode = 0;
  g.run = g.stop = nullptr;
  k_oz_gemm_group<S, BNT><<<grid, THREADS, smem_bytes<S, BNT>(), s>>>(ma, mb, g, grp);
  note_launch();
  return cudaGetLastError();
}

}  // namespace oz
}  // namespace sky
