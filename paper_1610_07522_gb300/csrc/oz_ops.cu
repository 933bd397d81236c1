// FP64 and FP32 forms of the overlap / Hamiltonian matrices (Eqs. normmatrix,
// hammatrix) and of the recombination psi = phi M (Sec. 3.3.3) on the tensor
// cores through the exact-integer split GEMM of oz_gemm.cuh.
//
// The split kernels work on the bit patterns only (integer exponent, mantissa
// and shifts; no FP64 arithmetic, which runs at 1/64 of the FP32 rate on this
// chip): each value x of a row with exponent E (|x| < 2^E over the row) is
// rounded to the integer X = round(|x| 2^{8S - E}) < 2^{8S} + 1 and written as
// balanced base-256 digits alpha_0 .. alpha_{S-1} (alpha_0 in [0, 256],
// the others in [-128, 127]), then given the sign of x (|alpha_s| <= 128).
//
// Complex contractions are real GEMMs over the interleaved (re, im) storage,
// as in the split-BF16 forms:
//   <a|b>:  Re = sum_k a_r[k] b_r[k],  Im = sum_k a_r[k] b'_r[k],
//           b' = (Im b, -Re b): D = a_r [b_r; b'_r]^T holds Re | Im;
//   psi_a = sum_b M[b][a] phi_b:  psi_r = [M_re^T | M_im^T] [phi_r; (i phi)_r],
//           the phi operand transposed (K = state index contiguous), rows v'
//           of the real view, both halves of K padded to round32(I).
#include <climits>
#include <cstdlib>

#include "oz_digits.cuh"
#include "oz_gemm.cuh"

namespace sky {

namespace {

using namespace ozdig;

// Device-side gate of a launch sequence (a problem whose iteration the device
// has stopped): skip the work when run says 0 or stop says non-zero.
__device__ __forceinline__ bool gated_off(const int* run, const int* stop) {
  return (run && *run == 0) || (stop && *stop != 0);
}

template <typename R>
__device__ __forceinline__ int block_max(int v) {
  __shared__ int red[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : INT_MIN;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (threadIdx.x == 0) red[0] = v;
  }
  __syncthreads();
  const int r = red[0];
  __syncthreads();
  return r;
}

// E[r] = exponent bound of row r of a [R][V] complex array (0 for a zero row).
template <typename T>
__global__ void __launch_bounds__(256) k_oz_rowexp(const T* __restrict__ src, long long V, int* E,
                                                   const int* run, const int* stop) {
  using R = decltype(T().x);
  if (gated_off(run, stop)) return;
  const T* row = src + (long long)blockIdx.x * V;
  int m = INT_MIN;
  for (long long k = threadIdx.x; k < V; k += blockDim.x) {
    const T v = row[k];
    m = max(m, max(exp_of((R)v.x), exp_of((R)v.y)));
  }
  m = block_max<R>(m);
  if (threadIdx.x == 0) E[blockIdx.x] = m == INT_MIN ? 0 : m;
}

// Slices of rows [0, R) of a [R][V] complex array over complex columns
// [c0, c0 + nc): dst[s][r][2 (c - c0) + {0, 1}]; with prime_off >= 0 also
// rows prime_off + r = (Im, -Re).
template <typename T, int S>
__global__ void __launch_bounds__(256) k_oz_split_rows(const T* __restrict__ src, int R, long long V,
                                                       long long c0, long long nc,
                                                       const int* __restrict__ E,
                                                       unsigned short* dst, long long ld,
                                                       long long ss, int prime_off,
                                                       const int* run, const int* stop) {
  using RT = decltype(T().x);
  if (gated_off(run, stop)) return;
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)R * nc) return;
  const int r = (int)(e / nc);
  const long long c = e - (long long)r * nc;
  const T v = src[(long long)r * V + c0 + c];
  const int Er = E[r];
  unsigned short dr[S], di[S];
  digits<S>((RT)v.x, Er, dr);
  digits<S>((RT)v.y, Er, di);
  unsigned* d32 = reinterpret_cast<unsigned*>(dst);
#pragma unroll
  for (int s = 0; s < S; ++s) {
    d32[(s * ss + (long long)r * ld) / 2 + c] = pack2(dr[s], di[s]);
    if (prime_off >= 0)
      d32[(s * ss + (long long)(prime_off + r) * ld) / 2 + c] = pack2(di[s], neg_bf16(dr[s]));
  }
}

// Row operand of the recombination: row a = [Re M[b][a] (b < I) | 0 | Im M[b][a] | 0],
// halves of Ipad; Ea[a] its exponent.  One block per row a.
template <int S>
__global__ void __launch_bounds__(256) k_oz_rot_a(const double2* __restrict__ M, int I, int Ipad,
                                                  unsigned short* dst, long long ld, long long ss,
                                                  int* Ea) {
  const int a = blockIdx.x;
  int m = INT_MIN;
  for (int b = threadIdx.x; b < I; b += blockDim.x) {
    const double2 v = M[(long long)b * I + a];
    m = max(m, max(exp_of(v.x), exp_of(v.y)));
  }
  m = block_max<double>(m);
  const int E = m == INT_MIN ? 0 : m;
  if (threadIdx.x == 0) Ea[a] = E;
  for (int b = threadIdx.x; b < Ipad; b += blockDim.x) {
    unsigned short dr[S], di[S];
    const double2 v = b < I ? M[(long long)b * I + a] : make_double2(0.0, 0.0);
    digits<S>(v.x, E, dr);
    digits<S>(v.y, E, di);
#pragma unroll
    for (int s = 0; s < S; ++s) {
      dst[s * ss + (long long)a * ld + b] = dr[s];
      dst[s * ss + (long long)a * ld + Ipad + b] = di[s];
    }
  }
}

// F[v] = exponent bound over the states of entry v (both parts) of [I][V].
template <typename T>
__global__ void __launch_bounds__(256) k_oz_colexp(const T* __restrict__ phi, int I, long long V,
                                                   int* F) {
  using R = decltype(T().x);
  const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= V) return;
  int m = INT_MIN;
  for (int b = 0; b < I; ++b) {
    const T x = phi[(long long)b * V + v];
    m = max(m, max(exp_of((R)x.x), exp_of((R)x.y)));
  }
  F[v] = m == INT_MIN ? 0 : m;
}

// Transposed operand of the recombination for complex columns [v0, v0 + nv):
// rows v' = 2 (v - v0) (+1), K index b' = b (phi_r) and Ipad + b ((i phi)_r):
//   row 2v:   Re phi_b[v],  -Im phi_b[v];   row 2v+1: Im phi_b[v],  Re phi_b[v];
// zeros for b in [I, Ipad).  32 states x 32 entries per block through shared
// memory (coalesced reads along v, writes along b).
template <typename T, int S>
__global__ void __launch_bounds__(256) k_oz_split_rot_b(const T* __restrict__ phi, int I, int Ipad,
                                                        long long V, long long v0, long long nv,
                                                        const int* __restrict__ F,
                                                        unsigned short* dst, long long ld,
                                                        long long ss) {
  using R = decltype(T().x);
  __shared__ T t[32][33];
  const int b0 = blockIdx.y * 32;
  const long long vb = (long long)blockIdx.x * 32;   // relative to v0
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8
  for (int r = ty; r < 32; r += 8) {
    const int b = b0 + r;
    const long long v = vb + tx;
    T z;
    z.x = 0; z.y = 0;
    t[r][tx] = (b < I && v < nv) ? phi[(long long)b * V + v0 + v] : z;
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const long long v = vb + r;   // entry handled by this warp; lanes run over states
    if (v >= nv) continue;
    const int b = b0 + tx;
    const T x = t[tx][r];
    const int Fv = F[v0 + v];
    unsigned short dr[S], di[S];
    digits<S>((R)x.x, Fv, dr);
    digits<S>((R)x.y, Fv, di);
#pragma unroll
    for (int s = 0; s < S; ++s) {
      unsigned short* row0 = dst + s * ss + (2 * v) * ld;
      unsigned short* row1 = row0 + ld;
      row0[b] = dr[s];
      row0[Ipad + b] = neg_bf16(di[s]);
      row1[b] = di[s];
      row1[Ipad + b] = dr[s];
    }
  }
}

// Digits of the rows of an n x n complex matrix operand in one pass per row
// (one block per row r): the operand row is row r of src, or with trans the
// conjugate of column r (a conjugate transpose read in place).  Its exponent
// goes to E[r]; digits to dst[s][r][2k + {0, 1}], and with prime_off >= 0
// (Im, -Re) to row prime_off + r.
template <int S>
__global__ void __launch_bounds__(256) k_oz_split_mat(const double2* __restrict__ src, int n,
                                                      int trans, int* E, unsigned short* dst,
                                                      long long ld, long long ss, int prime_off,
                                                      const int* run, const int* stop) {
  if (gated_off(run, stop)) return;
  const int r = blockIdx.x;
  auto at = [&](int k) {
    return trans ? conjx(src[(long long)k * n + r]) : src[(long long)r * n + k];
  };
  int m = INT_MIN;
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    const double2 v = at(k);
    m = max(m, max(exp_of(v.x), exp_of(v.y)));
  }
  m = block_max<double>(m);
  const int Er = m == INT_MIN ? 0 : m;
  if (threadIdx.x == 0) E[r] = Er;
  unsigned* d32 = reinterpret_cast<unsigned*>(dst);
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    const double2 v = at(k);
    unsigned short dr[S], di[S];
    digits<S>(v.x, Er, dr);
    digits<S>(v.y, Er, di);
#pragma unroll
    for (int s = 0; s < S; ++s) {
      d32[(s * ss + (long long)r * ld) / 2 + k] = pack2(dr[s], di[s]);
      if (prime_off >= 0)
        d32[(s * ss + (long long)(prime_off + r) * ld) / 2 + k] = pack2(di[s], neg_bf16(dr[s]));
    }
  }
}

// C[m][c] = conj(sum_z (P_z[m][c] + i P_z[m][n + c])) 2^{Ea[m] + Eb[c] - 16}: the
// product X Y from the full overlap of X with Zt = conj(Y)^T.
__global__ void k_oz_zgemm_reduce(const float2* __restrict__ P, int nz, long long sp, long long ldp,
                                  int n, const int* __restrict__ Ea, const int* __restrict__ Eb,
                                  double2* C, const int* run, const int* stop) {
  if (gated_off(run, stop)) return;
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)n * n) return;
  const int m = (int)(e / n), c = (int)(e % n);
  double re = 0.0, im = 0.0;
  for (int z = 0; z < nz; ++z) {
    const float2* Pz = P + z * sp + (long long)m * ldp;
    const float2 r = Pz[c], i = Pz[n + c];
    re += (double)r.x + (double)r.y;
    im += (double)i.x + (double)i.y;
  }
  const double sc = oz::pow2d(Ea[m] + Eb[c] - 16);
  C[e] = make_double2(sc * re, -sc * im);
}

// Grouped form of the two kernels above (blockIdx.y = problem b of the
// group; rows stacked at G.ra / G.rb, exponents indexed by stacked row).
// Operand B (second) adds the (Im, -Re) rows n .. 2n - 1 of its problem.
// Every row is written up to ld (zeros from K = 2n on), so a K block that
// runs past 2n reads zeros.
template <int S>
__global__ void __launch_bounds__(256) k_oz_split_group(oz::OzGroup G, int second, int trans,
                                                        int* E, unsigned short* dst, long long ld,
                                                        long long ss) {
  const int b = blockIdx.y, r = blockIdx.x;
  const int n = G.n[b];
  if (r >= n || oz::group_gated(G, b)) return;
  const double2* __restrict__ src = second ? G.B[b] : G.A[b];
  auto at = [&](int k) {
    return trans ? conjx(src[(long long)k * n + r]) : src[(long long)r * n + k];
  };
  int m = INT_MIN;
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    const double2 v = at(k);
    m = max(m, max(exp_of(v.x), exp_of(v.y)));
  }
  m = block_max<double>(m);
  const int Er = m == INT_MIN ? 0 : m;
  const long long row = (second ? G.rb[b] : G.ra[b]) + r;
  if (threadIdx.x == 0) E[row] = Er;
  unsigned* d32 = reinterpret_cast<unsigned*>(dst);
  const long long kh = ld / 2;   // complex entries per row, padding included
  for (int k = threadIdx.x; k < kh; k += blockDim.x) {
    unsigned short dr[S], di[S];
    if (k < n) {
      const double2 v = at(k);
      digits<S>(v.x, Er, dr);
      digits<S>(v.y, Er, di);
    } else {
#pragma unroll
      for (int s = 0; s < S; ++s) dr[s] = di[s] = 0;
    }
#pragma unroll
    for (int s = 0; s < S; ++s) {
      d32[(s * ss + row * ld) / 2 + k] = pack2(dr[s], di[s]);
      if (second) d32[(s * ss + (row + n) * ld) / 2 + k] = pack2(di[s], neg_bf16(dr[s]));
    }
  }
}

__global__ void k_oz_reduce_group(const float2* __restrict__ P, oz::OzGroup G,
                                  const int* __restrict__ Ea, const int* __restrict__ Eb) {
  const int b = blockIdx.y, n = G.n[b];
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)n * n || oz::group_gated(G, b)) return;
  const int m = (int)(e / n), c = (int)(e % n);
  const float2* Pm = P + G.po[b] + (long long)m * 2 * n;
  const float2 r = Pm[c], i = Pm[n + c];
  const double re = (double)r.x + (double)r.y, im = (double)i.x + (double)i.y;
  const double sc = oz::pow2d(Ea[G.ra[b] + m] + Eb[G.rb[b] + c] - 16);
  G.C[b][e] = make_double2(sc * re, -sc * im);
}

// X[a][b] (+)= dV 2^{Ea[a] + Eb[b] - 16} sum_z (P_z[a][b] + i P_z[a][I + b]) for a >= b
// (each P entry an unevaluated pair hi + lo), mirrored.
__global__ void k_oz_overlap_reduce(const float2* __restrict__ P, int nz, long long sp,
                                    long long ldp, int I, const int* __restrict__ Ea,
                                    const int* __restrict__ Eb, double dV, double2* X,
                                    int accumulate) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)I * I) return;
  const int a = (int)(e / I), b = (int)(e % I);
  if (a < b) return;
  double re = 0.0, im = 0.0;
  for (int z = 0; z < nz; ++z) {
    const float2* Pz = P + z * sp + (long long)a * ldp;
    const float2 r = Pz[b], i = Pz[I + b];
    re += (double)r.x + (double)r.y;
    im += (double)i.x + (double)i.y;
  }
  const double sc = dV * oz::pow2d(Ea[a] + Eb[b] - 16);
  double2 s = make_double2(sc * re, sc * im);
  if (accumulate) s = s + X[(long long)a * I + b];
  X[(long long)a * I + b] = s;
  if (a != b) X[(long long)b * I + a] = conjx(s);
}

inline int oz_slices(sky_prec p) { return p == SKY_F64 ? oz::kS64 : oz::kS32; }
inline int oz_bn(sky_prec p) { return p == SKY_F64 ? oz::kBN64 : oz::kBN32; }
inline long long round_up(long long x, long long m) { return (x + m - 1) / m * m; }

// K splits of the overlap GEMM: about one wave of items over the SMs, each
// split at least 8 K blocks (two exact segments).
int oz_overlap_splits(int I, long long K, int bn, int nsm) {
  const int tiles = oz::count_tiles(I, 2 * I, bn, true, I);
  const long long nkb = (K + oz::BK - 1) / oz::BK;
  long long z = (nsm + tiles - 1) / (tiles > 0 ? tiles : 1);
  const long long zmax = nkb / 8 > 0 ? nkb / 8 : 1;
  if (z > zmax) z = zmax;
  if (z < 1) z = 1;
  return (int)z;
}

template <int S, int BN>
sky_status oz_overlap_t(Ctx* c, const void* a, const void* b, int I, double2* X) {
  const long long V = 2LL * c->G;             // complex entries per state
  const bool f64 = c->prec == SKY_F64;
  int* Ea = c->d_ozE;
  int* Eb = c->d_ozE + c->max_states;
  cudaStream_t st = c->stream;
  // exponents over whole rows (shared by every K chunk)
  if (f64) {
    k_oz_rowexp<double2><<<I, 256, 0, st>>>((const double2*)a, V, Ea, nullptr, nullptr);
    if (b != a) k_oz_rowexp<double2><<<I, 256, 0, st>>>((const double2*)b, V, Eb, nullptr, nullptr);
  } else {
    k_oz_rowexp<float2><<<I, 256, 0, st>>>((const float2*)a, V, Ea, nullptr, nullptr);
    if (b != a) k_oz_rowexp<float2><<<I, 256, 0, st>>>((const float2*)b, V, Eb, nullptr, nullptr);
  }
  note_launch(b != a ? 2 : 1);
  if (b == a) Eb = Ea;
  // K chunk (complex entries) so that S slices of the 2I B rows fit the buffer
  long long nc = c->oz_b_elems / ((long long)S * 2 * I) / 2;
  nc = nc / 64 * 64;   // whole 128-value segments
  if (nc > V) nc = V;
  if (nc < 64 && nc < V) return set_err(c, SKY_EINVAL, "overlap: split buffer too small for I=%d", I);
  const long long ldp = 2LL * I;
  bool first = true;
  for (long long c0 = 0; c0 < V; c0 += nc) {
    const long long n = (V - c0) < nc ? (V - c0) : nc;
    const long long K = 2 * n, ld = round_up(K, 8);
    unsigned short* Bp = (unsigned short*)c->d_ozB;
    unsigned short* Ap = (unsigned short*)c->d_ozA;
    const long long sb = (long long)2 * I * ld, sa = (long long)I * ld;
    const long long tot = (long long)I * n;
    if (f64) {
      k_oz_split_rows<double2, S><<<div_up(tot, 256), 256, 0, st>>>(
          (const double2*)b, I, V, c0, n, Eb, Bp, ld, sb, I, nullptr, nullptr);
      if (b != a)
        k_oz_split_rows<double2, S><<<div_up(tot, 256), 256, 0, st>>>(
            (const double2*)a, I, V, c0, n, Ea, Ap, ld, sa, -1, nullptr, nullptr);
    } else {
      k_oz_split_rows<float2, S><<<div_up(tot, 256), 256, 0, st>>>(
          (const float2*)b, I, V, c0, n, Eb, Bp, ld, sb, I, nullptr, nullptr);
      if (b != a)
        k_oz_split_rows<float2, S><<<div_up(tot, 256), 256, 0, st>>>(
            (const float2*)a, I, V, c0, n, Ea, Ap, ld, sa, -1, nullptr, nullptr);
    }
    note_launch(b != a ? 2 : 1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_check(c, e, "oz split");
    int z = oz_overlap_splits(I, K, BN, c->num_sms);
    const long long spart = (long long)I * ldp;
    if ((size_t)z * spart > c->oz_p_elems) z = (int)(c->oz_p_elems / spart);
    if (z < 1) return set_err(c, SKY_EINVAL, "overlap: partial buffer too small for I=%d", I);
    oz::OzArgs g{};
    g.mode = 0;
    g.P = c->d_ozP;
    g.ldp = ldp;
    g.sp = spart;
    g.status = c->d_status;
    const void* Aop = b != a ? (const void*)Ap : (const void*)Bp;
    const long long lda = ld, sA = b != a ? sa : sb;
    e = oz::oz_gemm<S, BN>(Aop, lda, sA, I, Bp, ld, sb, 2 * I, (int)K, true, I, g, &z, st);
    if (e != cudaSuccess) return cuda_check(c, e, "oz overlap gemm");
    k_oz_overlap_reduce<<<div_up((long long)I * I, 256), 256, 0, st>>>(
        c->d_ozP, z, spart, ldp, I, Ea, Eb, c->dV, X, first ? 0 : 1);
    note_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_check(c, e, "oz overlap reduce");
    first = false;
  }
  return SKY_OK;
}

template <int S, int BN>
sky_status oz_rotate_t(Ctx* c, const void* phi, const double2* M, int I, void* out) {
  const long long V = 2LL * c->G;
  const bool f64 = c->prec == SKY_F64;
  const int Ipad = (int)round_up(I, 32);
  const long long ldk = 2LL * Ipad;
  cudaStream_t st = c->stream;
  int* Ea = c->d_ozE;
  int* F = c->d_ozE + c->max_states;
  unsigned short* Ap = (unsigned short*)c->d_ozA;
  unsigned short* Bp = (unsigned short*)c->d_ozB;
  const long long sa = (long long)I * ldk;
  if ((long long)S * sa > (long long)c->oz_a_elems)
    return set_err(c, SKY_EINVAL, "rotate: split buffer too small for I=%d", I);
  k_oz_rot_a<S><<<I, 256, 0, st>>>(M, I, Ipad, Ap, ldk, sa, Ea);
  if (f64) k_oz_colexp<double2><<<div_up(V, 256), 256, 0, st>>>((const double2*)phi, I, V, F);
  else k_oz_colexp<float2><<<div_up(V, 256), 256, 0, st>>>((const float2*)phi, I, V, F);
  note_launch(2);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_check(c, e, "oz rotate split a");
  // complex columns per chunk so that S slices of 2 nv rows fit the buffer
  long long nv = c->oz_b_elems / ((long long)S * 2 * ldk);
  nv = nv / 480 * 480;   // 2 nv rows: a multiple of both tile widths
  if (nv > V) nv = V;
  if (nv < 480 && nv < V) return set_err(c, SKY_EINVAL, "rotate: split buffer too small for I=%d", I);
  for (long long v0 = 0; v0 < V; v0 += nv) {
    const long long n = (V - v0) < nv ? (V - v0) : nv;
    const long long sb = 2 * n * ldk;
    dim3 g2(div_up(n, 32), Ipad / 32);
    if (f64)
      k_oz_split_rot_b<double2, S><<<g2, 256, 0, st>>>((const double2*)phi, I, Ipad, V, v0, n, F,
                                                       Bp, ldk, sb);
    else
      k_oz_split_rot_b<float2, S><<<g2, 256, 0, st>>>((const float2*)phi, I, Ipad, V, v0, n, F, Bp,
                                                      ldk, sb);
    note_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_check(c, e, "oz rotate split b");
    oz::OzArgs g{};
    g.mode = 1;
    g.out = f64 ? (void*)((double*)out + 2 * v0) : (void*)((float*)out + 2 * v0);
    g.ldo = 2 * V;
    g.out_f32 = f64 ? 0 : 1;
    g.ea = Ea;
    g.eb = F + v0;
    g.eb_shift = 1;
    g.status = c->d_status;
    int z = 1;
    e = oz::oz_gemm<S, BN>(Ap, ldk, sa, I, Bp, ldk, sb, (int)(2 * n), (int)ldk, false, I, g, &z,
                           st);
    if (e != cudaSuccess) return cuda_check(c, e, "oz rotate gemm");
  }
  return SKY_OK;
}

}  // namespace

// C = opA(A) opB(B) for n x n complex FP64 matrices (op: identity or conjugate
// transpose) on the tensor cores: with X = opA(A) and Zt = conj(opB(B))^T,
// C[m][c] = conj(sum_k conj(X[m][k]) Zt[c][k]), the full digit-split overlap
// of X's rows with Zt's rows (6 digits; about 1e-14 of the largest element).
// Every kernel is skipped when the device gate (run, stop) says so.
bool oz_zgemm_fits(const Ctx* c, int n) {
  // the digit rows are written with the padded stride ld = round_up(2n, 8)
  const long long ld = round_up(2LL * n, 8);
  return c->d_ozB && n <= c->max_states &&
         (long long)oz::kS64 * 2 * n * ld <= (long long)c->oz_b_elems &&
         (long long)oz::kS64 * n * ld <= (long long)c->oz_a_elems;
}

sky_status oz_zgemm(Ctx* c, bool ah, bool bh, const double2* A, const double2* B, double2* C,
                    int n, const int* run, const int* stop) {
  constexpr int S = oz::kS64, BN = oz::kBN64;
  cudaStream_t st = c->stream;
  int* Ea = c->d_ozE;
  int* Eb = c->d_ozE + c->max_states;
  const long long K = 2LL * n, ld = round_up(K, 8);
  unsigned short* Bp = (unsigned short*)c->d_ozB;
  unsigned short* Ap = (unsigned short*)c->d_ozA;
  const long long sb = 2LL * n * ld, sa = (long long)n * ld;
  const long long tot = (long long)n * n;
  // X = opA(A): rows of A, or conjugated columns; Zt = conj(opB(B))^T: rows of
  // B when opB is the conjugate transpose, else conjugated columns of B
  k_oz_split_mat<S><<<n, 256, 0, st>>>(A, n, ah ? 1 : 0, Ea, Ap, ld, sa, -1, run, stop);
  k_oz_split_mat<S><<<n, 256, 0, st>>>(B, n, bh ? 0 : 1, Eb, Bp, ld, sb, n, run, stop);
  note_launch(2);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_check(c, e, "oz zgemm split");
  const int tiles = oz::count_tiles(n, 2 * n, BN, false, n);
  const long long nkb = (K + oz::BK - 1) / oz::BK;
  long long z = (c->num_sms + tiles - 1) / tiles;
  if (z > nkb / 8) z = nkb / 8;
  if (z < 1) z = 1;
  const long long spart = 2LL * n * n;
  if ((size_t)z * spart > c->oz_p_elems) z = (long long)(c->oz_p_elems / spart);
  if (z < 1) return set_err(c, SKY_EINVAL, "zgemm: partial buffer too small for n=%d", n);
  int zi = (int)z;
  oz::OzArgs g{};
  g.mode = 0;
  g.P = c->d_ozP;
  g.ldp = 2LL * n;
  g.sp = spart;
  g.status = c->d_status;
  g.run = run;
  g.stop = stop;
  e = oz::oz_gemm<S, BN>(Ap, ld, sa, n, Bp, ld, sb, 2 * n, (int)K, false, n, g, &zi, st);
  if (e != cudaSuccess) return cuda_check(c, e, "oz zgemm");
  k_oz_zgemm_reduce<<<div_up(tot, 256), 256, 0, st>>>(c->d_ozP, zi, spart, 2LL * n, n, Ea, Eb, C,
                                                      run, stop);
  note_launch();
  return cuda_check(c, cudaGetLastError(), "oz zgemm reduce");
}

// The products C_b = opA(A_b) opB(B_b) of every problem of a batch (n_b <=
// the context's state count) in one grouped launch sequence: two digit
// splits, one tensor-core launch over all problems' tiles, one reduction
// (the per-problem form above, stacked; gates per problem).
int oz_group_slices() { return oz::kS64; }

bool oz_zgemm_group_fits(const Ctx* c, int np, const int* n) {
  if (!c->d_ozgA || np > c->ozg_np) return false;
  long long rows = 0;
  long long p = 0;
  for (int b = 0; b < np; ++b) {
    if (n[b] > c->max_states) return false;
    rows += n[b];
    p += 2LL * n[b] * n[b];
  }
  return rows <= c->ozg_rows && p <= (long long)c->ozg_p_elems;
}

sky_status oz_zgemm_group(Ctx* c, const ZJobs& j) {
  constexpr int S = oz::kS64, BN = oz::kBN64;
  cudaStream_t st = c->stream;
  oz::OzGroup G;
  G.np = j.np;
  G.tile0[0] = 0;
  int ra = 0, nmax = 0;
  long long po = 0;
  for (int b = 0; b < j.np; ++b) {
    const int n = j.n[b];
    G.n[b] = n; G.ra[b] = ra; G.rb[b] = 2 * ra; G.po[b] = po;
    G.A[b] = j.A[b]; G.B[b] = j.B[b]; G.C[b] = j.C[b];
    G.run[b] = j.run[b]; G.stop[b] = j.stop[b];
    G.tile0[b + 1] = G.tile0[b] + (n > 0 ? ((n + oz::BM - 1) / oz::BM) * ((2 * n + BN - 1) / BN) : 0);
    ra += n;
    po += 2LL * n * n;
    nmax = n > nmax ? n : nmax;
  }
  if (nmax == 0) return SKY_OK;
  const long long ld = c->ozg_ld;
  const long long sa = (long long)c->ozg_rows * ld, sb = 2 * sa;
  int* Ea = c->d_ozgE;
  int* Eb = c->d_ozgE + c->ozg_rows;
  unsigned short* Ap = (unsigned short*)c->d_ozgA;
  unsigned short* Bp = (unsigned short*)c->d_ozgB;
  k_oz_split_group<S><<<dim3(nmax, j.np), 256, 0, st>>>(G, 0, j.ah ? 1 : 0, Ea, Ap, ld, sa);
  k_oz_split_group<S><<<dim3(nmax, j.np), 256, 0, st>>>(G, 1, j.bh ? 0 : 1, Eb, Bp, ld, sb);
  note_launch(2);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_check(c, e, "grouped zgemm split");
  oz::OzArgs g{};
  g.P = c->d_ozgP;
  g.status = c->d_status;
  e = oz::oz_gemm_group<S, BN>(Ap, sa, ra, Bp, sb, 2 * ra, ld, G, g, st);
  if (e != cudaSuccess) return cuda_check(c, e, "grouped zgemm");
  k_oz_reduce_group<<<dim3(div_up((long long)nmax * nmax, 256), j.np), 256, 0, st>>>(
      c->d_ozgP, G, Ea, Eb);
  note_launch();
  return cuda_check(c, cudaGetLastError(), "grouped zgemm reduce");
}

sky_status oz_overlap(Ctx* c, const void* a, const void* b, int I, double2* X) {
  if (c->prec == SKY_F64) return oz_overlap_t<oz::kS64, oz::kBN64>(c, a, b, I, X);
  return oz_overlap_t<oz::kS32, oz::kBN32>(c, a, b, I, X);
}

sky_status oz_rotate(Ctx* c, const void* phi, const double2* M, int I, void* out) {
  if (c->prec == SKY_F64) return oz_rotate_t<oz::kS64, oz::kBN64>(c, phi, M, I, out);
  return oz_rotate_t<oz::kS32, oz::kBN32>(c, phi, M, I, out);
}

// Slice buffers (bf16 elements over all slices), exponents and partials of
// the split GEMMs for up to Imax states of V complex entries.  The B buffer
// holds the [b; b'] overlap operand (or a K chunk of it) and the transposed
// recombination operand (or a chunk of its rows); its size is capped by
// SKY_OZ_MB (default 4096 MiB).
void oz_scratch_sizes(sky_prec prec, int Imax, long long V, int nsm, size_t* a_elems,
                      size_t* b_elems, size_t* e_elems, size_t* p_elems) {
  if (Imax <= 0 || V <= 0) {
    *a_elems = *b_elems = *e_elems = *p_elems = 1;
    return;
  }
  const int S = oz_slices(prec), bn = oz_bn(prec);
  const long long Ipad = round_up(Imax, 32);
  const long long ov_b = (long long)S * 2 * Imax * round_up(2 * V, 8);
  const long long rot_b = (long long)S * 2 * V * 2 * Ipad;
  long long need_b = ov_b > rot_b ? ov_b : rot_b;
  long long cap = 4096;
  if (const char* s = getenv("SKY_OZ_MB"))
    if (atol(s) > 0) cap = atol(s);
  cap = (cap << 20) / 2;
  // at least one chunk of 64 complex columns (overlap) / 480 (recombination)
  const long long min_b = (long long)S * 2 * Imax * 128 > (long long)S * 960 * 2 * Ipad
                              ? (long long)S * 2 * Imax * 128
                              : (long long)S * 960 * 2 * Ipad;
  if (need_b > cap) need_b = cap > min_b ? cap : min_b;
  *b_elems = (size_t)need_b;
  // A: the a rows of an overlap chunk (at most half of B) or the rotation rows
  const long long rot_a = (long long)S * Imax * 2 * Ipad;
  *a_elems = (size_t)(need_b / 2 > rot_a ? need_b / 2 : rot_a);
  *e_elems = (size_t)(2 * Imax + V + 64);
  size_t pmax = 1;
  for (int I = 1; I <= Imax; ++I) {
    const size_t p = (size_t)oz_overlap_splits(I, 2 * V, bn, nsm) * I * 2 * I;
    if (p > pmax) pmax = p;
  }
  *p_elems = pmax;
}

}  // namespace sky
