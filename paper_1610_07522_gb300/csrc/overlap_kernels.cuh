// Overlap-matrix kernels X = <a|b> (Eqs. normmatrix, hammatrix), lower
// triangle only (Fig. 3), split along the contraction index V.  Shared by
// sky_overlap and sky_overlap_noalloc.
#pragma once

#include "sky_internal.cuh"

namespace sky {

constexpr int BM = 32, BN = 32, BK = 16;   // tile of 32 x 32 complex outputs

__device__ __forceinline__ double2 ld2(const double2* p) { return *p; }
__device__ __forceinline__ double2 ld2(const float2* p) { const float2 v = *p; return make_double2(v.x, v.y); }

// acc += conj(a) b and acc += a b as four FMAs each.
__device__ __forceinline__ void cfma_conj(double2& acc, double2 a, double2 b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(-a.y, b.x, acc.y);
}
__device__ __forceinline__ void cfma(double2& acc, double2 a, double2 b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
}

// ---------------------------------------------------------------- overlap
// Lower-triangle tile t -> (ti, tj), ti >= tj.
__device__ __forceinline__ void tri_tile(int t, int& ti, int& tj) {
  int i = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
  while ((i + 1) * (i + 2) / 2 <= t) ++i;
  while (i * (i + 1) / 2 > t) --i;
  ti = i;
  tj = t - i * (i + 1) / 2;
}

// part[split][a][b] = sum_{v in split} conj(A[a][v]) Bm[b][v] for the lower
// tiles (FULL: for every tile, blockIdx.x = ti * ntile + tj).
// Three real products per complex multiply-add (Gauss):
//   P1 = sum a.x b.x,  P2 = sum a.y b.y,  P3 = sum (a.x - a.y)(b.x + b.y),
//   Re = P1 + P2,  Im = P3 - P1 + P2;
// the sums a.x - a.y and b.x + b.y are formed once when staging the tile.
template <typename S, bool FULL = false>
__global__ void __launch_bounds__(256) k_overlap(const S* __restrict__ A, const S* __restrict__ Bm,
                                                 int I, long long V, long long kchunk,
                                                 double2* __restrict__ part) {
  __shared__ double2 As[BK][BM + 1];
  __shared__ double2 Bs[BK][BN + 1];
  __shared__ double Ad[BK][BM + 1];
  __shared__ double Bd[BK][BN + 1];
  int ti, tj;
  if (FULL) {
    const int nt = (I + BM - 1) / BM;
    ti = blockIdx.x / nt;
    tj = blockIdx.x % nt;
  } else {
    tri_tile(blockIdx.x, ti, tj);
  }
  const int r0 = ti * BM, c0 = tj * BN;
  const long long kb = (long long)blockIdx.y * kchunk;
  const long long ke = (kb + kchunk) < V ? (kb + kchunk) : V;
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  const int lrow = tid >> 3, lk = (tid & 7) * 2;   // loader: 32 rows x 16 k
  double p1[2][2], p2[2][2], p3[2][2];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) p1[i][j] = p2[i][j] = p3[i][j] = 0.0;
  for (long long k0 = kb; k0 < ke; k0 += BK) {
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const long long k = k0 + lk + u;
      const int ra = r0 + lrow, rb = c0 + lrow;
      const double2 av = (ra < I && k < ke) ? ld2(A + (long long)ra * V + k) : make_double2(0.0, 0.0);
      const double2 bv = (rb < I && k < ke) ? ld2(Bm + (long long)rb * V + k) : make_double2(0.0, 0.0);
      As[lk + u][lrow] = av;
      Ad[lk + u][lrow] = av.x - av.y;
      Bs[lk + u][lrow] = bv;
      Bd[lk + u][lrow] = bv.x + bv.y;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      double2 a[2], b[2];
      double ad[2], bd[2];
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        a[i] = As[kk][ty * 2 + i];
        ad[i] = Ad[kk][ty * 2 + i];
        b[i] = Bs[kk][tx * 2 + i];
        bd[i] = Bd[kk][tx * 2 + i];
      }
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          p1[i][j] = fma(a[i].x, b[j].x, p1[i][j]);
          p2[i][j] = fma(a[i].y, b[j].y, p2[i][j]);
          p3[i][j] = fma(ad[i], bd[j], p3[i][j]);
        }
    }
    __syncthreads();
  }
  double2* dst = part + (long long)blockIdx.y * I * I;
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int r = r0 + ty * 2 + i, cc = c0 + tx * 2 + j;
      if (r < I && cc < I && (FULL || r >= cc))
        dst[(long long)r * I + cc] = make_double2(p1[i][j] + p2[i][j], p3[i][j] - p1[i][j] + p2[i][j]);
    }
}

// X[a][b] = dV sum_split part (a >= b); X[b][a] = conj(X[a][b]).
static __global__ void k_overlap_reduce(const double2* part, int nsplit, int I, double dV, double2* X) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)I * I) return;
  const int a = (int)(e / I), b = (int)(e % I);
  if (a < b) return;
  double2 s = make_double2(0.0, 0.0);
  for (int k = 0; k < nsplit; ++k) s = s + part[(long long)k * I * I + e];
  s = dV * s;
  X[(long long)a * I + b] = s;
  if (a != b) X[(long long)b * I + a] = conjx(s);
}

// X[a][b] = dV sum_split part for every (a, b).
static __global__ void k_overlap_reduce_full(const double2* part, int nsplit, int I, double dV,
                                             double2* X) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)I * I) return;
  double2 s = make_double2(0.0, 0.0);
  for (int k = 0; k < nsplit; ++k) s = s + part[(long long)k * I * I + e];
  X[e] = dV * s;
}

}  // namespace sky
