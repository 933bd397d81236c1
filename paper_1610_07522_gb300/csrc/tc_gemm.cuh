// BF16 tensor-core GEMM for sm_103a with 5th-generation tensor cores:
//   D[m][n] (fp32) = sum_k A[m][k] B[n][k]          (A, B bf16, K contiguous)
// summed over up to six (A_i, B_j) operand pairs ("phases"), which is how the
// split-BF16 products (hi*hi + hi*lo + lo*hi for a 2-way split, six products
// for a 3-way split) accumulate in one tile.
//
// Persistent kernel, one CTA per SM: CTA b computes the 128 x BNT output tiles
// b, b + gridDim.x, ... (m fastest, then n, then the K split; split z writes
// partial tile z).  Each ring stage holds one 64-wide K block of every operand
// piece in use (A_0..A_{n-1}, B_0..B_{n-1}), so a piece is loaded once per K
// block and all products of that block are issued from the same stage.  Two
// TMEM accumulators alternate between tiles, so the epilogue of one tile runs
// while the MMAs of the next are issued.  Warp roles:
//   warp 0     TMA producer: cp.async.bulk.tensor loads of 128 x 64 bf16
//              A and B boxes (128-byte swizzle) into a ring of a.stages stages,
//              running ahead across tile boundaries;
//   warp 1     owns TMEM (2 x BNT fp32 columns) and one elected lane issues
//              tcgen05.mma (M = 128, N = BNT, K = 16 each); tcgen05.commit frees
//              ring stages and signals the epilogue when a tile is complete;
//   warps 2-5  epilogue: tcgen05.ld of their TMEM lane quadrant -> global fp32,
//              then hand the accumulator back (one mbarrier arrival per warp).
// Every mbarrier wait is bounded; a timeout sets SKY_ETIMEOUT in the status
// word, the kernel waits (bounded) for the MMAs it issued, frees TMEM and
// returns.
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>

#include "sky_internal.cuh"

namespace sky {
namespace tc {

constexpr int BM = 128, BN = 128, BK = 64;         // BK bf16 = one 128-byte swizzle row
constexpr int TILE_BYTES = BM * BK * 2;            // 16 KiB per 128-row operand tile
// BN: the 128-column tile used for sizing (partial tiles, tile counts of callers);
// the kernel also runs with 256-column tiles (template BNT), see gemm_bf16.
constexpr int kMaxStages = 8;
constexpr int kRingBytes = 200 * 1024;             // ring budget (of 227 KB)
constexpr int SMEM_BYTES = kRingBytes + 1024 + 256;
constexpr int THREADS = 192;
// TMEM: two accumulators (double buffer) of BNT fp32 columns each
constexpr long long kSpin = 1LL << 24;             // x >= 64 ns per try: bounded waits

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for the phase with the given parity to complete.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (long long i = 0; i < kSpin; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if (i > 256) __nanosleep(64);
  }
  return false;
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int c0, int c1,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"((unsigned long long)map), "r"(c0), "r"(c1), "r"(bar)
      : "memory");
}
// Shared-memory matrix descriptor: K-major tile with 128-byte swizzle, rows of
// 128 bytes, 8-row groups 1024 bytes apart (stride byte offset), tcgen05
// descriptor version 1, layout type 2 (128B swizzle).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | (1ull << 16) | (64ull << 32) | (1ull << 46) |
         (2ull << 61);
}
// Instruction descriptor, kind::f16: D fp32, A and B bf16, both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(da), "l"(db), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
      : "memory");
}
__device__ __forceinline__ void fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// 32 consecutive fp32 columns of this warp's 32 TMEM lanes (one row per lane).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
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
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

constexpr int kMaxPhase = 6;

struct GemmArgs {
  int M, N, K;              // K in bf16 elements
  int kb_per_split;         // 64-wide K blocks per split (blockIdx.z)
  int nphase;               // phases: sum_p A[pa[p]] B[pb[p]]^T
  int pa[kMaxPhase], pb[kMaxPhase];
  int npiece;               // pieces of each operand loaded per stage
  int stages;               // ring depth (stage = 2 npiece tiles)
  int nsplit;               // K splits (tiles are m x n x split)
  float* D;                 // D[z][m][n], row stride ldd, split stride sstride
  long long ldd, sstride;
  int* status;
};

template <int BNT>
__global__ void __launch_bounds__(THREADS, 1)
    k_gemm_bf16(const __grid_constant__ CUtensorMap mA0, const __grid_constant__ CUtensorMap mA1,
                const __grid_constant__ CUtensorMap mA2, const __grid_constant__ CUtensorMap mB0,
                const __grid_constant__ CUtensorMap mB1, const __grid_constant__ CUtensorMap mB2,
                GemmArgs a) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base =
      (unsigned char*)(((unsigned long long)smem_raw + 1023ull) & ~1023ull);
  constexpr int TILE_B = BNT * BK * 2;              // bytes of one B piece tile
  constexpr uint32_t TMEM_COLS = 2 * BNT;
  const int np = a.npiece, stages = a.stages;
  const int stage_bytes = np * (TILE_BYTES + TILE_B);
  unsigned long long* bars = (unsigned long long*)(base + kRingBytes);
  uint32_t* tmem_slot = (uint32_t*)(bars + 2 * kMaxStages + 5);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // persistent: CTA b takes tiles b, b + gridDim.x, ...; tile t -> (m fastest, n, split)
  const int mt = (a.M + BM - 1) / BM, nt = (a.N + BNT - 1) / BNT;
  const int ntiles = mt * nt * a.nsplit;
  const int nkb_total = (a.K + BK - 1) / BK;
  auto tile_kb = [&](int t, int& m0, int& n0, int& kb0, int& nkb, int& z) {
    m0 = (t % mt) * BM;
    n0 = ((t / mt) % nt) * BNT;
    z = t / (mt * nt);
    kb0 = z * a.kb_per_split;
    nkb = nkb_total - kb0;
    if (nkb > a.kb_per_split) nkb = a.kb_per_split;
    if (nkb < 0) nkb = 0;
  };
  const uint32_t bar0 = smem_u32(bars);
  auto full = [&](int s) { return bar0 + 8u * s; };
  auto empty = [&](int s) { return bar0 + 8u * (kMaxStages + s); };
  auto acc_full = [&](int b) { return bar0 + 8u * (2 * kMaxStages + b); };
  auto acc_empty = [&](int b) { return bar0 + 8u * (2 * kMaxStages + 2 + b); };
  const uint32_t drain = bar0 + 8u * (2 * kMaxStages + 4);

  if (threadIdx.x == 0) {
    for (int s = 0; s < stages; ++s) {
      mbar_init(full(s), 1);
      mbar_init(empty(s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(acc_full(b), 1);
      mbar_init(acc_empty(b), 4);   // one arrival per epilogue warp
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
      // stage layout: A_0 .. A_{np-1}, B_0 .. B_{np-1}, one 16 KiB tile each
      long long g = 0;   // ring position across all tiles of this CTA
      bool ok = true;
      for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
        int m0, n0, kb0, nkb, z;
        tile_kb(t, m0, n0, kb0, nkb, z);
        for (int it = 0; it < nkb; ++it, ++g) {
          const int s = (int)(g % stages);
          const long long u = g / stages;
          if (u > 0 && !mbar_wait(empty(s), (uint32_t)((u - 1) & 1))) {
            flag_status(a.status, SKY_ETIMEOUT);
            ok = false;
            break;
          }
          const int kb = kb0 + it;
          const uint32_t sa = smem_u32(base + s * stage_bytes);
          mbar_expect_tx(full(s), stage_bytes);
          for (int i = 0; i < np; ++i) {
            const CUtensorMap* mapA = i == 0 ? &mA0 : (i == 1 ? &mA1 : &mA2);
            const CUtensorMap* mapB = i == 0 ? &mB0 : (i == 1 ? &mB1 : &mB2);
            tma_load_2d(sa + i * TILE_BYTES, mapA, kb * BK, m0, full(s));
            tma_load_2d(sa + np * TILE_BYTES + i * TILE_B, mapB, kb * BK, n0, full(s));
          }
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16(BM, BNT);
      long long g = 0;
      int j = 0;   // tiles done by this CTA
      bool ok = true;
      for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++j) {
        int m0, n0, kb0, nkb, z;
        tile_kb(t, m0, n0, kb0, nkb, z);
        const int b = j & 1, use = j >> 1;
        // the epilogue must have drained this accumulator's previous tile
        if (use > 0 && !mbar_wait(acc_empty(b), (uint32_t)((use - 1) & 1))) {
          flag_status(a.status, SKY_ETIMEOUT);
          break;
        }
        fence_after();
        const uint32_t acc = tmem + (uint32_t)(b * BNT);
        for (int it = 0; it < nkb; ++it, ++g) {
          const int s = (int)(g % stages);
          const long long u = g / stages;
          if (!mbar_wait(full(s), (uint32_t)(u & 1))) {
            flag_status(a.status, SKY_ETIMEOUT);
            ok = false;
            break;
          }
          fence_after();
          const uint32_t sa = smem_u32(base + s * stage_bytes);
          for (int p = 0; p < a.nphase; ++p) {
            const uint64_t da = sw128_desc(sa + a.pa[p] * TILE_BYTES);
            const uint64_t db = sw128_desc(sa + np * TILE_BYTES + a.pb[p] * TILE_B);
#pragma unroll
            for (int k = 0; k < BK / 16; ++k)   // +32 bytes along K = +2 in the encoded address
              mma_bf16(acc, da + 2ull * k, db + 2ull * k, idesc,
                       (it > 0 || p > 0 || k > 0) ? 1u : 0u);
          }
          mma_commit(empty(s));
        }
        mma_commit(acc_full(b));   // arrives when this tile's MMAs have completed
      }
      // every MMA issued by this thread completes before TMEM is freed
      mma_commit(drain);
      if (!mbar_wait(drain, 0)) flag_status(a.status, SKY_ETIMEOUT);
    }
  } else {
    // epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 of the tile's accumulator
    const int q = warp & 3;
    int j = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++j) {
      int m0, n0, kb0, nkb, z;
      tile_kb(t, m0, n0, kb0, nkb, z);
      const int b = j & 1, use = j >> 1;
      const bool ok = mbar_wait(acc_full(b), (uint32_t)(use & 1));
      if (!ok) {
        if (lane == 0) flag_status(a.status, SKY_ETIMEOUT);
        break;
      }
      fence_after();
      const int row = m0 + q * 32 + lane;
      float* drow = a.D + (long long)z * a.sstride + (long long)row * a.ldd;
#pragma unroll 1
      for (int c = 0; c < BNT; c += 32) {
        float v[32];
        tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * BNT + c), v);
        if (nkb == 0) {
#pragma unroll
          for (int i = 0; i < 32; ++i) v[i] = 0.0f;
        }
        const int col = n0 + c;
        if (row < a.M) {
          if (col + 32 <= a.N) {
#pragma unroll
            for (int i = 0; i < 32; i += 4)
              *reinterpret_cast<float4*>(drow + col + i) =
                  make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
          } else {
            for (int i = 0; i < 32 && col + i < a.N; ++i) drow[col + i] = v[i];
          }
        }
      }
      // this warp's lanes of the accumulator are read: hand it back to the MMA warp
      fence_before();
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(acc_empty(b)) : "memory");
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

// ---------------------------------------------------------------- host side
// bf16 matrix [rows][K] with row stride ld (elements, multiple of 8), K-major.
inline cudaError_t make_map(CUtensorMap* map, const void* ptr, int rows, int K, long long ld,
                            int box_rows) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                     cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
    encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
  }
  const cuuint64_t gdim[2] = {(cuuint64_t)K, (cuuint64_t)rows};
  const cuuint64_t gstride[1] = {(cuuint64_t)ld * 2};
  const cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
  const cuuint32_t estride[2] = {1, 1};
  CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), gdim,
                      gstride, box, estride, CU_TENSOR_MAP_INTERLEAVE_NONE,
                      CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// Products of a split-BF16 operand pair: the terms kept of
// (A0 + A1 + A2)(B0 + B1 + B2)^T, by decreasing weight.
struct Phases {
  int n;
  int pa[kMaxPhase], pb[kMaxPhase];
};
inline Phases phases_for_split(int nsplit) {
  Phases p;
  if (nsplit == 1) {
    p.n = 1; p.pa[0] = 0; p.pb[0] = 0;
  } else if (nsplit == 2) {          // hi*hi + hi*lo + lo*hi
    p.n = 3;
    const int a[3] = {0, 0, 1}, b[3] = {0, 1, 0};
    for (int i = 0; i < 3; ++i) { p.pa[i] = a[i]; p.pb[i] = b[i]; }
  } else {                            // all products of weight <= 2 of a 3-way split
    p.n = 6;
    const int a[6] = {0, 0, 1, 0, 1, 2}, b[6] = {0, 1, 0, 2, 1, 0};
    for (int i = 0; i < 6; ++i) { p.pa[i] = a[i]; p.pb[i] = b[i]; }
  }
  return p;
}

// D = sum over phases of A[pa] B[pb]^T.  A[i]: [M][K], B[i]: [N][K] bf16 with
// row strides lda, ldb >= K (elements, multiples of 8), i < nsplit.  With *splits > 1
// the K blocks are divided over blockIdx.z and partial tiles go to
// D + z * sstride; *splits returns the number of partial tiles written.
// Pointers 16-byte aligned, ldd a multiple of 4.
inline cudaError_t gemm_bf16(const void* const* A, long long lda, const void* const* B,
                             long long ldb, int nsplit, int M, int N, int K, int* splits,
                             float* D, long long ldd, long long sstride, int* status,
                             cudaStream_t s, int tile_n = 0) {
  if (M <= 0 || N <= 0 || K <= 0) { *splits = 0; return cudaSuccess; }
  // TMA needs 16-byte row strides; columns past K read as zeros
  if ((lda & 7) || (ldb & 7) || (ldd & 3) || lda < K || ldb < K || nsplit < 1 || nsplit > 3)
    return cudaErrorInvalidValue;
  // 128 x 256 tiles when the pieces of one K block still fit twice in the ring
  // (x3: 96 KiB per stage), else 128 x 128 (x6: 96 KiB per stage); tile_n
  // 128 asks for the narrow tiles (more tiles, for products that share the GPU)
  const int bnt = (nsplit <= 2 && (long long)N >= 256 && tile_n != 128) ? 256 : 128;
  CUtensorMap ma[3], mb[3];
  cudaError_t e;
  for (int i = 0; i < 3; ++i) {
    const int j = i < nsplit ? i : 0;
    if ((e = make_map(&ma[i], A[j], M, K, lda, BM)) != cudaSuccess) return e;
    if ((e = make_map(&mb[i], B[j], N, K, ldb, bnt)) != cudaSuccess) return e;
  }
  const Phases ph = phases_for_split(nsplit);
  const int nkb = (K + BK - 1) / BK;
  int stages = kRingBytes / (nsplit * (TILE_BYTES + bnt * BK * 2));
  if (stages > kMaxStages) stages = kMaxStages;
  int z = *splits < 1 ? 1 : *splits;
  if (z > nkb) z = nkb;
  GemmArgs g;
  g.M = M; g.N = N; g.K = K;
  g.kb_per_split = (nkb + z - 1) / z;
  z = (nkb + g.kb_per_split - 1) / g.kb_per_split;
  g.nphase = ph.n;
  g.npiece = nsplit;
  g.stages = stages;
  for (int i = 0; i < kMaxPhase; ++i) {
    g.pa[i] = i < ph.n ? ph.pa[i] : 0;
    g.pb[i] = i < ph.n ? ph.pb[i] : 0;
  }
  g.D = D; g.ldd = ldd; g.sstride = sstride; g.status = status;
  // the shared-memory opt-ins are set once per device (before any stream capture)
  static bool smem_set[64] = {false};
  int dev = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (!smem_set[dev]) {
    e = cudaFuncSetAttribute(k_gemm_bf16<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_gemm_bf16<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
    if (e != cudaSuccess) return e;
    smem_set[dev] = true;
  }
  g.nsplit = z;
  const long long ntiles = (long long)((M + BM - 1) / BM) * ((N + bnt - 1) / bnt) * z;
  int nsm = 0;
  if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  const int grid = (int)(ntiles < nsm ? ntiles : nsm);   // persistent: one CTA per SM
  if (bnt == 256)
    k_gemm_bf16<256><<<grid, THREADS, SMEM_BYTES, s>>>(ma[0], ma[1], ma[2], mb[0], mb[1], mb[2], g);
  else
    k_gemm_bf16<128><<<grid, THREADS, SMEM_BYTES, s>>>(ma[0], ma[1], ma[2], mb[0], mb[1], mb[2], g);
  note_launch();
  *splits = z;
  return cudaGetLastError();
}

}  // namespace tc
}  // namespace sky
