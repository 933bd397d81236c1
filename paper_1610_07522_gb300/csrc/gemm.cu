// Complex contractions of step 3 (Sec. 3.3): the overlap and Hamiltonian
// matrices X = <a|b> (Eqs. normmatrix, hammatrix; lower triangle only, as in
// Fig. 3), the recombination psi = phi M (Sec. 3.3.3) and small I x I
// products for the Loewdin and Rayleigh-Ritz factors.  FP64 FMA on the CUDA
// cores; FP32 spinors are widened on load.  The FP64 and FP32 forms send the
// overlap and the recombination to the tensor-core split GEMMs of oz_ops.cu
// unless SKY_KNOB_SPLIT_GEMM is 0.
#include "overlap_kernels.cuh"

namespace sky {

// K-splits so that tiles x splits fills whole waves of resident CTAs
// (`slots` = CTAs resident on the GPU at once), capped by the K blocks.
static int overlap_splits(int I, long long V, int slots, int* ntiles_out) {
  const int nt = (I + BM - 1) / BM;
  const int ntiles = nt * (nt + 1) / 2;
  const long long kblocks = (V + BK - 1) / BK;
  long long want = slots / ntiles;
  if (want < 1) want = 1;
  if (want > kblocks) want = kblocks;
  if (ntiles_out) *ntiles_out = ntiles;
  return (int)want;
}

int overlap_slots(int num_sms) {
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_overlap<double2>, 256, 0);
  if (per_sm < 1) per_sm = 1;
  return per_sm * num_sms;
}

size_t overlap_partial_elems(int I, long long V, int slots) {
  return (size_t)overlap_splits(I, V, slots, nullptr) * (size_t)I * (size_t)I;
}

sky_status overlap_impl(Ctx* c, const void* a, const void* b, int I, double2* X) {
  if (is_tc(c->prec)) return tc_overlap(c, a, b, I, X);
  if (c->oz_on) return oz_overlap(c, a, b, I, X);
  const long long V = 2LL * c->G;
  int ntiles;
  const int nsplit = overlap_splits(I, V, c->ov_waves * c->ov_slots, &ntiles);
  const long long kblocks = (V + BK - 1) / BK;
  const long long kchunk = ((kblocks + nsplit - 1) / nsplit) * BK;
  const int nsplit_eff = (int)((V + kchunk - 1) / kchunk);
  if ((size_t)nsplit_eff * I * I > c->gpart_elems)
    return set_err(c, SKY_EINVAL, "overlap scratch too small for I=%d", I);
  dim3 grid(ntiles, nsplit_eff);
  if (c->prec == SKY_F64)
    k_overlap<double2><<<grid, 256, 0, c->stream>>>((const double2*)a, (const double2*)b, I, V,
                                                    kchunk, c->d_gpart);
  else
    k_overlap<float2><<<grid, 256, 0, c->stream>>>((const float2*)a, (const float2*)b, I, V,
                                                   kchunk, c->d_gpart);
  note_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_check(c, e, "overlap");
  k_overlap_reduce<<<div_up((long long)I * I, 256), 256, 0, c->stream>>>(c->d_gpart, nsplit_eff, I,
                                                                       c->dV, X); note_launch();
  return cuda_check(c, cudaGetLastError(), "overlap reduce");
}

// Full X = <a|b> for two different state sets (no Hermitian mirror), FP64
// accumulation in every precision: split-K like overlap_impl.
sky_status cross_overlap_impl(Ctx* c, const void* a, const void* b, int I, double2* X) {
  const long long V = 2LL * c->G;
  const int nt = (I + BM - 1) / BM;
  const int ntiles = nt * nt;
  const long long kblocks = (V + BK - 1) / BK;
  long long want = c->ov_slots / ntiles;
  if (want < 1) want = 1;
  if (want > kblocks) want = kblocks;
  const long long kchunk = ((kblocks + want - 1) / want) * BK;
  const int nsplit = (int)((V + kchunk - 1) / kchunk);
  if ((size_t)nsplit * I * I > c->gpart_elems)
    return set_err(c, SKY_EINVAL, "cross overlap scratch too small for I=%d", I);
  dim3 grid(ntiles, nsplit);
  if (c->prec == SKY_F64)
    k_overlap<double2, true><<<grid, 256, 0, c->stream>>>((const double2*)a, (const double2*)b, I, V,
                                                          kchunk, c->d_gpart);
  else
    k_overlap<float2, true><<<grid, 256, 0, c->stream>>>((const float2*)a, (const float2*)b, I, V,
                                                         kchunk, c->d_gpart);
  note_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_check(c, e, "cross overlap");
  k_overlap_reduce_full<<<div_up((long long)I * I, 256), 256, 0, c->stream>>>(c->d_gpart, nsplit, I,
                                                                            c->dV, X); note_launch();
  return cuda_check(c, cudaGetLastError(), "cross overlap reduce");
}

// ---------------------------------------------------------------- rotate
// out[a][v] = sum_b M[b][a] phi[b][v]; tile rows a (32) x columns v (32).
// Three real products per complex multiply-add (Gauss):
//   P1 = sum m.x f.x,  P2 = sum m.y f.y,  P3 = sum (m.x + m.y)(f.x + f.y),
//   Re = P1 - P2,  Im = P3 - P1 - P2.
template <typename S>
__global__ void __launch_bounds__(256) k_rotate(const S* __restrict__ phi, const double2* __restrict__ M,
                                                int I, long long V, S* __restrict__ out) {
  __shared__ double2 As[BK][BM + 1];
  __shared__ double2 Bs[BK][BN + 1];
  __shared__ double Ad[BK][BM + 1];
  __shared__ double Bd[BK][BN + 1];
  const int r0 = blockIdx.y * BM;
  const long long v0 = (long long)blockIdx.x * BN;
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  double p1[2][2], p2[2][2], p3[2][2];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) p1[i][j] = p2[i][j] = p3[i][j] = 0.0;
  for (int k0 = 0; k0 < I; k0 += BK) {
    // 16 k x 32 entries per operand, 2 per thread, contiguous along the tile row
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int e = tid * 2 + u;
      const int kk = e >> 5, col = e & 31;
      const int k = k0 + kk;
      const int a = r0 + col;
      const long long v = v0 + col;
      const double2 mv = (k < I && a < I) ? M[(long long)k * I + a] : make_double2(0.0, 0.0);
      const double2 fv = (k < I && v < V) ? ld2(phi + (long long)k * V + v) : make_double2(0.0, 0.0);
      As[kk][col] = mv;
      Ad[kk][col] = mv.x + mv.y;
      Bs[kk][col] = fv;
      Bd[kk][col] = fv.x + fv.y;
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
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int r = r0 + ty * 2 + i;
      const long long v = v0 + tx * 2 + j;
      if (r < I && v < V) {
        const double re = p1[i][j] - p2[i][j], im = p3[i][j] - p1[i][j] - p2[i][j];
        if constexpr (std::is_same<S, double2>::value)
          out[(long long)r * V + v] = make_double2(re, im);
        else
          out[(long long)r * V + v] = make_float2((float)re, (float)im);
      }
    }
}

sky_status rotate_impl(Ctx* c, const void* phi, const double2* M, int I, void* out) {
  if (is_tc(c->prec)) return tc_rotate(c, phi, M, I, out);
  if (c->oz_on) return oz_rotate(c, phi, M, I, out);
  const long long V = 2LL * c->G;
  dim3 grid(div_up(V, BN), div_up(I, BM));
  if (c->prec == SKY_F64)
    k_rotate<double2><<<grid, 256, 0, c->stream>>>((const double2*)phi, M, I, V, (double2*)out);
  else
    k_rotate<float2><<<grid, 256, 0, c->stream>>>((const float2*)phi, M, I, V, (float2*)out);
  note_launch();
  return cuda_check(c, cudaGetLastError(), "rotate");
}

// ---------------------------------------------------------------- small GEMMs
// C[b] = opA(A[b]) opB(B[b]) for a batch of n[b] x n[b] row-major products
// (op = identity or conjugate transpose), blockIdx.z = problem.  TS x TS output
// tile per block, 2 x 2 per thread.  Problem b runs only if run[b] is null or
// *run[b] != 0, and stop[b] is null or *stop[b] == 0 (device-side gating, so a
// fixed launch sequence can skip work the device decided is not needed).
ZJobs zjobs(int np, bool ah, bool bh, const double2* const* A, const double2* const* B,
            double2* const* C, const int* n, const int* const* run, const int* const* stop) {
  ZJobs j;
  j.np = np; j.ah = ah; j.bh = bh;
  for (int b = 0; b < kMaxBatch; ++b) {
    const bool in = b < np;
    j.A[b] = in ? A[b] : nullptr;
    j.B[b] = in ? B[b] : nullptr;
    j.C[b] = in ? C[b] : nullptr;
    j.n[b] = in ? n[b] : 0;
    j.run[b] = in ? run[b] : nullptr;
    j.stop[b] = in ? stop[b] : nullptr;
  }
  return j;
}

// Three real products per complex multiply-add (Gauss), as in k_overlap:
//   P1 = sum a.x b.x,  P2 = sum a.y b.y,  P3 = sum (a.x + a.y)(b.x + b.y),
//   Re = P1 - P2,  Im = P3 - P1 - P2;
// the sums a.x + a.y and b.x + b.y are formed once when staging the tiles
// (after the conjugation of a conjugate-transposed operand).
template <bool AH, bool BH, int TS>
__global__ void __launch_bounds__(TS * TS / 4) k_zgemm(ZJobs j) {
  const int b = blockIdx.z, n = j.n[b];
  const int r0 = blockIdx.y * TS, c0 = blockIdx.x * TS;
  if (r0 >= n || c0 >= n) return;
  if ((j.run[b] && *j.run[b] == 0) || (j.stop[b] && *j.stop[b] != 0)) return;
  const double2* __restrict__ A = j.A[b];
  const double2* __restrict__ B = j.B[b];
  constexpr int NT = TS * TS / 4, TH = TS / 2;
  __shared__ double2 As[BK][TS + 1];
  __shared__ double2 Bs[BK][TS + 1];
  __shared__ double Ad[BK][TS + 1];
  __shared__ double Bd[BK][TS + 1];
  const int tid = threadIdx.x, ty = tid / TH, tx = tid % TH;
  double p1[2][2], p2[2][2], p3[2][2];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int k = 0; k < 2; ++k) p1[i][k] = p2[i][k] = p3[i][k] = 0.0;
  for (int k0 = 0; k0 < n; k0 += BK) {
    for (int e = tid; e < BK * TS; e += NT) {
      const int kk = e / TS, col = e % TS;
      const int k = k0 + kk, r = r0 + col, cc = c0 + col;
      double2 av = make_double2(0.0, 0.0), bv = make_double2(0.0, 0.0);
      if (k < n && r < n) av = AH ? conjx(A[(long long)k * n + r]) : A[(long long)r * n + k];
      if (k < n && cc < n) bv = BH ? conjx(B[(long long)cc * n + k]) : B[(long long)k * n + cc];
      As[kk][col] = av;
      Ad[kk][col] = av.x + av.y;
      Bs[kk][col] = bv;
      Bd[kk][col] = bv.x + bv.y;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      double2 a[2], bb[2];
      double ad[2], bd[2];
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        a[i] = As[kk][ty * 2 + i];
        ad[i] = Ad[kk][ty * 2 + i];
        bb[i] = Bs[kk][tx * 2 + i];
        bd[i] = Bd[kk][tx * 2 + i];
      }
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int k = 0; k < 2; ++k) {
          p1[i][k] = fma(a[i].x, bb[k].x, p1[i][k]);
          p2[i][k] = fma(a[i].y, bb[k].y, p2[i][k]);
          p3[i][k] = fma(ad[i], bd[k], p3[i][k]);
        }
    }
    __syncthreads();
  }
  double2* C = j.C[b];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const int r = r0 + ty * 2 + i, cc = c0 + tx * 2 + k;
      if (r < n && cc < n)
        C[(long long)r * n + cc] = make_double2(p1[i][k] - p2[i][k], p3[i][k] - p1[i][k] - p2[i][k]);
    }
}

template <int TS>
static void launch_zgemm(Ctx* c, const ZJobs& j, int nmax) {
  dim3 grid(div_up(nmax, TS), div_up(nmax, TS), j.np);
  constexpr int NT = TS * TS / 4;
  if (!j.ah && !j.bh) k_zgemm<false, false, TS><<<grid, NT, 0, c->stream>>>(j);
  else if (j.ah && !j.bh) k_zgemm<true, false, TS><<<grid, NT, 0, c->stream>>>(j);
  else if (!j.ah && j.bh) k_zgemm<false, true, TS><<<grid, NT, 0, c->stream>>>(j);
  else k_zgemm<true, true, TS><<<grid, NT, 0, c->stream>>>(j);
}

sky_status zgemm_batch(Ctx* c, const ZJobs& jin) {
  // a batch of many problems: every product in one grouped tensor-core launch
  // sequence (oz_zgemm_group), when its buffers hold them
  if (jin.np > kOzGroupMin && oz_zgemm_group_fits(c, jin.np, jin.n)) return oz_zgemm_group(c, jin);
  // problems of kOzZgemmMin states or more: tensor-core digit-split products
  // (one launch sequence each, gated like the rest); the others in one
  // batched FP64 launch
  ZJobs j = jin;
  for (int b = 0; b < j.np; ++b) {
    const bool gated = j.run[b] || j.stop[b];
    if (j.n[b] >= (gated ? kOzZgemmGated : kOzZgemmMin) && oz_zgemm_fits(c, j.n[b])) {
      const sky_status s = oz_zgemm(c, j.ah, j.bh, j.A[b], j.B[b], j.C[b], j.n[b], j.run[b], j.stop[b]);
      if (s != SKY_OK) return s;
      j.n[b] = 0;
    }
  }
  int nmax = 0;
  long long tiles32 = 0;
  for (int b = 0; b < j.np; ++b) {
    if (j.n[b] > nmax) nmax = j.n[b];
    tiles32 += (long long)div_up(j.n[b], 32) * div_up(j.n[b], 32);
  }
  if (nmax == 0) return SKY_OK;
  // 32 x 32 tiles once they give at least two blocks per SM, else 16 x 16
  if (tiles32 >= 2LL * c->num_sms) launch_zgemm<32>(c, j, nmax);
  else launch_zgemm<16>(c, j, nmax);
  note_launch();
  return cuda_check(c, cudaGetLastError(), "zgemm");
}

sky_status zgemm_small(Ctx* c, bool ah, bool bh, const double2* A, const double2* B, double2* C,
                       int n, const int* run, const int* stop) {
  return zgemm_batch(c, zjobs(1, ah, bh, &A, &B, &C, &n, &run, &stop));
}

}  // namespace sky
