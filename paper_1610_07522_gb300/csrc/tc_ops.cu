// Split-BF16 tensor-core forms of the overlap / Hamiltonian matrix (Eqs.
// normmatrix, hammatrix) and of the recombination (Sec. 3.3.3) for FP32
// spinors.  Each FP32 value x is split into bf16 pieces x = x_0 + x_1 (+ x_2)
// with x_0 = bf16(x), x_1 = bf16(x - x_0), x_2 = bf16(x - x_0 - x_1); the
// products kept are those of total weight <= nsplit - 1 (3 products for a
// 2-way split, 6 for a 3-way split), accumulated in FP32 in TMEM.
//
// Complex contractions become single real GEMMs over the interleaved (re, im)
// storage:
//   <a|b>:  Re = sum_k a_r[k] b_r[k],  Im = sum_k a_r[k] b'_r[k],
//           b' = (Im b, -Re b) per entry, so D = a_r [b_r; b'_r]^T holds Re | Im;
//   psi_a = sum_b M[b][a] phi_b:  psi_r = [M_re^T | M_im^T] [phi_r; (i phi)_r],
//           i phi = (-Im phi, Re phi), with the phi operand stored transposed
//           (K contiguous: the two halves padded with zeros to a multiple of 32
//           states each) so that D = psi_r directly.
#include <cuda_bf16.h>

#include "tc_gemm.cuh"

namespace sky {

__device__ __forceinline__ void split3(float x, int n, __nv_bfloat16* out) {
  const __nv_bfloat16 h = __float2bfloat16_rn(x);
  out[0] = h;
  if (n > 1) {
    const float r = x - __bfloat162float(h);
    const __nv_bfloat16 m = __float2bfloat16_rn(r);
    out[1] = m;
    if (n > 2) out[2] = __float2bfloat16_rn(r - __bfloat162float(m));
  }
}

// Row operands of <a|b>: dst[i][row][k] for the real view of src ([rows][K]);
// with prime != 0, rows [rows, 2 rows) receive (Im, -Re) of each entry.
__global__ void k_split_rows(const float* __restrict__ src, long long rows, long long K, int n,
                             int prime, __nv_bfloat16* d0, __nv_bfloat16* d1, __nv_bfloat16* d2) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;   // complex entry
  const long long nc = rows * (K / 2);
  if (e >= nc) return;
  const long long r = e / (K / 2), c = e % (K / 2);
  __nv_bfloat16 sr[3], si[3];
  split3(src[2 * e], n, sr);
  split3(src[2 * e + 1], n, si);
  __nv_bfloat16* d[3] = {d0, d1, d2};
  for (int i = 0; i < n; ++i) {
    __nv_bfloat162 v;
    v.x = sr[i]; v.y = si[i];
    *reinterpret_cast<__nv_bfloat162*>(d[i] + r * K + 2 * c) = v;
    if (prime) {
      __nv_bfloat162 w;
      w.x = si[i]; w.y = __hneg(sr[i]);
      *reinterpret_cast<__nv_bfloat162*>(d[i] + (rows + r) * K + 2 * c) = w;
    }
  }
}

// Transposed operand of the recombination: dst[i][v'][beta'] (row stride ld)
// from phi_r[beta][v'] (beta' = beta) and (i phi)_r (beta' = Ipad + beta), with
// zeros for beta in [I, Ipad); Ipad a multiple of 32.  32 x 32 tiles through
// shared memory (coalesced on both sides, whole 32-byte sectors written).
__global__ void __launch_bounds__(256) k_split_rot_b(const float* __restrict__ phi, int I,
                                                     int Ipad, long long K2V, long long ld, int n,
                                                     __nv_bfloat16* d0, __nv_bfloat16* d1,
                                                     __nv_bfloat16* d2) {
  __shared__ float t[32][65];    // [beta][v' (32 complex = 64 reals)]
  const int b0 = blockIdx.y * 32;
  const long long v0 = (long long)blockIdx.x * 64;        // real index
  const int tx = threadIdx.x & 63, ty = threadIdx.x >> 6;  // 64 x 4
  for (int r = ty; r < 32; r += 4) {
    const int b = b0 + r;
    const long long v = v0 + tx;
    t[r][tx] = (b < I && v < K2V) ? phi[(long long)b * K2V + v] : 0.0f;
  }
  __syncthreads();
  __nv_bfloat16* d[3] = {d0, d1, d2};
  // write: each thread one (v', beta) pair; beta fastest for coalescing
  for (int idx = threadIdx.x; idx < 64 * 32; idx += 256) {
    const int vl = idx >> 5, bl = idx & 31;
    const long long v = v0 + vl;
    const int b = b0 + bl;
    if (v >= K2V) continue;
    const float x = t[bl][vl];            // zero for b >= I
    // (i phi)_r: even v' (re slot) takes -Im, odd v' (im slot) takes +Re
    const float y = (vl & 1) ? t[bl][vl - 1] : -t[bl][vl + 1];
    __nv_bfloat16 sx[3], sy[3];
    split3(x, n, sx);
    split3(y, n, sy);
    for (int i = 0; i < n; ++i) {
      d[i][v * ld + b] = sx[i];
      d[i][v * ld + Ipad + b] = sy[i];
    }
  }
}

// Row operand of the recombination: A[alpha][beta'] = M_re[beta'][alpha]
// (beta' < I) or M_im[beta' - I][alpha], split into bf16 pieces.
__global__ void k_split_rot_a(const double2* __restrict__ M, int I, int Ipad, long long ld, int n,
                              __nv_bfloat16* d0, __nv_bfloat16* d1, __nv_bfloat16* d2) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)I * 2 * Ipad) return;
  const int a = (int)(e / (2 * Ipad)), bp = (int)(e % (2 * Ipad));
  const int beta = bp < Ipad ? bp : bp - Ipad;
  // row a: [Re M[beta][a] for beta < I | zeros | Im M[beta][a] | zeros]
  double xd = 0.0;
  if (beta < I) {
    const double2 m = M[(long long)beta * I + a];
    xd = bp < Ipad ? m.x : m.y;   // the FP64 value keeps its residual in the lower pieces
  }
  __nv_bfloat16 s[3];
  const __nv_bfloat16 h = __double2bfloat16(xd);
  s[0] = h;
  if (n > 1) {
    const double r = xd - (double)__bfloat162float(h);
    const __nv_bfloat16 mm = __double2bfloat16(r);
    s[1] = mm;
    if (n > 2) s[2] = __double2bfloat16(r - (double)__bfloat162float(mm));
  }
  __nv_bfloat16* d[3] = {d0, d1, d2};
  for (int i = 0; i < n; ++i) d[i][(long long)a * ld + bp] = s[i];
}

// X[a][b] = dV sum_z (D_z[a][b] + i D_z[a][I + b]) for a >= b, mirrored.
__global__ void k_tc_overlap_reduce(const float* __restrict__ D, int nz, long long sstride,
                                    long long ldd, int I, double dV, double2* X) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)I * I) return;
  const int a = (int)(e / I), b = (int)(e % I);
  if (a < b) return;
  double re = 0.0, im = 0.0;
  for (int z = 0; z < nz; ++z) {
    const float* Dz = D + z * sstride + (long long)a * ldd;
    re += Dz[b];
    im += Dz[I + b];
  }
  const double2 s = make_double2(dV * re, dV * im);
  X[(long long)a * I + b] = s;
  if (a != b) X[(long long)b * I + a] = conjx(s);
}

// K layout of the recombination: [re | zeros | im | zeros] in halves of
// round32(I), so that both halves of each row start on a 64-byte boundary and
// every 32-byte sector of the transposed operand is written whole.
static inline long long round32(long long x) { return (x + 31) / 32 * 32; }

int tc_nsplit(sky_prec p) { return p == SKY_F32_BF16X6 ? 3 : 2; }

// FP32 accumulation in TMEM loses accuracy over long K (its rounding error
// grows like sqrt(K) 2^-24 of the partial sums): every split-K partial of the
// overlap covers at most kMaxAccK values of K, and the partials are summed in
// FP64 by the reduce.
constexpr long long kMaxAccK = 2048;
int tc_min_splits(long long K) { return (int)((K + kMaxAccK - 1) / kMaxAccK); }

// Scratch (bf16 elements per piece / fp32 partials) for I states of V complex.
void tc_scratch_sizes(int I, long long V, int num_sms, size_t* piece_a, size_t* piece_b,
                      size_t* piece_rot_a, size_t* partial) {
  const long long K = 2 * V;
  *piece_a = (size_t)I * K;
  const size_t ov_b = (size_t)2 * I * K;
  const size_t rot_b = (size_t)K * 2 * round32(I);
  *piece_b = ov_b > rot_b ? ov_b : rot_b;
  *piece_rot_a = (size_t)I * 2 * round32(I);
  const long long ldd = (2LL * I + 3) / 4 * 4;
  const int tiles = ((I + tc::BM - 1) / tc::BM) * ((2 * I + tc::BN - 1) / tc::BN);
  int z = kMaxTcWaves * num_sms / (tiles > 0 ? tiles : 1);
  const int zacc = tc_min_splits(K);
  if (z < zacc) z = zacc;
  if (z < 1) z = 1;
  *partial = (size_t)z * I * ldd;
}

sky_status tc_overlap(Ctx* c, const void* a, const void* b, int I, double2* X) {
  const long long V = 2LL * c->G, K = 2 * V;
  const int n = tc_nsplit(c->prec);
  __nv_bfloat16* A[3] = {(__nv_bfloat16*)c->d_tcA[0], (__nv_bfloat16*)c->d_tcA[1],
                         (__nv_bfloat16*)c->d_tcA[2]};
  __nv_bfloat16* Bp[3] = {(__nv_bfloat16*)c->d_tcB[0], (__nv_bfloat16*)c->d_tcB[1],
                          (__nv_bfloat16*)c->d_tcB[2]};
  const long long nc = (long long)I * V;
  k_split_rows<<<div_up(nc, 256), 256, 0, c->stream>>>((const float*)a, I, K, n, 0, A[0], A[1],
                                                       A[2]);
  k_split_rows<<<div_up(nc, 256), 256, 0, c->stream>>>((const float*)b, I, K, n, 1, Bp[0], Bp[1],
                                                       Bp[2]);
  note_launch(2);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_check(c, e, "tc split");
  const long long ldd = (2LL * I + 3) / 4 * 4;
  const int tiles = ((I + tc::BM - 1) / tc::BM) * ((2 * I + tc::BN - 1) / tc::BN);
  // tc_waves 0: the fewest splits the accumulation bound allows (for boxes
  // that share the GPU with others), else about that many waves of SMs
  int z = c->tc_waves * c->num_sms / tiles;
  if (z < tc_min_splits(K)) z = tc_min_splits(K);   // bounded FP32 accumulation length
  if (z < 1) z = 1;
  const long long sstride = (long long)I * ldd;
  if ((size_t)z * sstride > c->tc_partial_elems) z = (int)(c->tc_partial_elems / sstride);
  const void* pa[3] = {A[0], A[1], A[2]};
  const void* pb[3] = {Bp[0], Bp[1], Bp[2]};
  e = tc::gemm_bf16(pa, K, pb, K, n, I, 2 * I, (int)K, &z, c->d_tcPart, ldd, sstride,
                    c->d_status, c->stream, c->tc_tile_n);
  if (e != cudaSuccess) return cuda_check(c, e, "tc overlap gemm");
  k_tc_overlap_reduce<<<div_up((long long)I * I, 256), 256, 0, c->stream>>>(
      c->d_tcPart, z, sstride, ldd, I, c->dV, X);
  note_launch();
  return cuda_check(c, cudaGetLastError(), "tc overlap reduce");
}

sky_status tc_rotate(Ctx* c, const void* phi, const double2* M, int I, void* out) {
  const long long V = 2LL * c->G, K2V = 2 * V;
  const int n = tc_nsplit(c->prec);
  const int Ipad = (int)round32(I);
  const long long ldk = 2LL * Ipad;
  __nv_bfloat16* Ra[3] = {(__nv_bfloat16*)c->d_tcRotA[0], (__nv_bfloat16*)c->d_tcRotA[1],
                          (__nv_bfloat16*)c->d_tcRotA[2]};
  __nv_bfloat16* Bp[3] = {(__nv_bfloat16*)c->d_tcB[0], (__nv_bfloat16*)c->d_tcB[1],
                          (__nv_bfloat16*)c->d_tcB[2]};
  k_split_rot_a<<<div_up((long long)I * 2 * Ipad, 256), 256, 0, c->stream>>>(M, I, Ipad, ldk, n,
                                                                            Ra[0], Ra[1], Ra[2]);
  dim3 g2(div_up(K2V, 64), Ipad / 32);
  k_split_rot_b<<<g2, 256, 0, c->stream>>>((const float*)phi, I, Ipad, K2V, ldk, n, Bp[0], Bp[1],
                                           Bp[2]);
  note_launch(2);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_check(c, e, "tc rotate split");
  int z = 1;
  const void* pa[3] = {Ra[0], Ra[1], Ra[2]};
  const void* pb[3] = {Bp[0], Bp[1], Bp[2]};
  e = tc::gemm_bf16(pa, ldk, pb, ldk, n, I, (int)K2V, 2 * Ipad, &z, (float*)out, K2V, 0,
                    c->d_status, c->stream, c->tc_tile_n);
  return cuda_check(c, e, "tc rotate gemm");
}

}  // namespace sky
