// Single-particle Hamiltonian (Sec. 2.1-2.2), damped gradient step
// (Eq. dampstep) and densities (Eqs. rho, curr, tau) for batched spinors.
//
// h psi is evaluated in the rearranged but identical form
//   h psi = U psi - (i/2) sum_j A_j (d_j psi) + sum_j d_j F_j,
//   F_j   = -B d_j psi - (i/2) A_j psi,   A_j = (sigma x W)_j,
// which follows from eps_ijk W_i sigma_k = (sigma x W)_j.  The passes are
//   1. G_j = d_j psi               (one 1D spectral pass per axis)
//   2. L = U psi - (i/2) sum A_j G_j -> hpsi;  F_j -> in place of G_j
//   3. F_j <- d_j F_j              (one pass per axis, in place)
//   4. hpsi = L + sum_j F_j, with <psi|h psi> and |h psi|^2 per block.
#include "fft_lines.cuh"

namespace sky {

sky_status upload_twiddles_hamiltonian(Ctx* c) {
  return cuda_check(c, upload_twiddles_this_unit(), "twiddle upload (hamiltonian)");
}

// ------------------------------------------------------------ line ops
// out = d_axis in  (i (k + theta/L) / N after the forward transform)
template <typename T> struct OpDeriv {
  static constexpr bool kFwd = true, kInv = true;
  const cx<T>* in; cx<T>* out; const T* k; T inv_n; long long G;
  __device__ __forceinline__ cx<T> load(long long b, int i) const { return in[b * G + i]; }
  __device__ __forceinline__ void mid(cx<T>& v, long long, int, int m) const {
    const T kk = k[m] * inv_n;
    v = mkc<T>(-kk * v.y, kk * v.x);
  }
  __device__ __forceinline__ void store(long long b, int i, cx<T> v) const { out[b * G + i] = v; }
};

// The same derivative pass of FP64 arrays with the transform carried in
// double-float arithmetic (dd.cuh): loads and stores FP64, k from a table of
// float pairs of (k + theta/L) / N.
struct OpDerivDD {
  static constexpr bool kFwd = true, kInv = true;
  const double2* in; double2* out; const float2* k; long long G;
  __device__ __forceinline__ ddc load(long long b, int i) const { return ddc_of(in[b * G + i]); }
  __device__ __forceinline__ void mid(ddc& v, long long, int, int m) const {
    const float2 kk = k[m];
    const dd kd(kk.x, kk.y);
    v = ddc{-(kd * v.y), kd * v.x};
  }
  __device__ __forceinline__ void store(long long b, int i, ddc v) const { out[b * G + i] = dbl2_of(v); }
};

// Damped step, z pass: r = hpsi - eps psi, forward along z, into phi.
template <typename T> struct OpDampZFwd {
  static constexpr bool kFwd = true, kInv = false;
  const cx<T>* psi; const cx<T>* hpsi; const double* eps; cx<T>* phi; long long G;
  __device__ __forceinline__ cx<T> load(long long b, int i) const {
    const T e = (T)eps[b >> 1];
    const cx<T> h = hpsi[b * G + i], p = psi[b * G + i];
    return mkc<T>(h.x - e * p.x, h.y - e * p.y);
  }
  __device__ __forceinline__ void mid(cx<T>&, long long, int, int) const {}
  __device__ __forceinline__ void store(long long b, int i, cx<T> v) const { phi[b * G + i] = v; }
};
// Plain forward or inverse pass in place.
template <typename T, bool INV> struct OpPass {
  static constexpr bool kFwd = !INV, kInv = INV;
  cx<T>* a; long long G;
  __device__ __forceinline__ cx<T> load(long long b, int i) const { return a[b * G + i]; }
  __device__ __forceinline__ void mid(cx<T>&, long long, int, int) const {}
  __device__ __forceinline__ void store(long long b, int i, cx<T> v) const { a[b * G + i] = v; }
};
// Damped step, x pass: forward, times x0 / (G (E0 + T(k))), inverse.
template <typename T> struct OpDampX {
  static constexpr bool kFwd = true, kInv = true;
  cx<T>* a; const double* P; T scale; long long G;
  __device__ __forceinline__ cx<T> load(long long b, int i) const { return a[b * G + i]; }
  __device__ __forceinline__ void mid(cx<T>& v, long long, int i, int) const {
    const T f = (T)P[i] * scale;
    v = mkc<T>(f * v.x, f * v.y);
  }
  __device__ __forceinline__ void store(long long b, int i, cx<T> v) const { a[b * G + i] = v; }
};
// Damped step, z pass: inverse along z, phi = psi - w(r) result (w = 1 when
// no per-voxel weight is given).
template <typename T> struct OpDampZInv {
  static constexpr bool kFwd = false, kInv = true;
  const cx<T>* psi; cx<T>* phi; const float* w; long long G;
  __device__ __forceinline__ cx<T> load(long long b, int i) const { return phi[b * G + i]; }
  __device__ __forceinline__ void mid(cx<T>&, long long, int, int) const {}
  __device__ __forceinline__ void store(long long b, int i, cx<T> v) const {
    if (w) {
      const T s = (T)w[i];
      v = mkc<T>(s * v.x, s * v.y);
    }
    phi[b * G + i] = psi[b * G + i] - v;
  }
};

template <typename T> const T* kt_of(const Ctx* c, int axis);
template <> const double* kt_of<double>(const Ctx* c, int axis) { return c->d_kt[axis]; }
template <> const float* kt_of<float>(const Ctx* c, int axis) { return c->d_ktf[axis]; }

// G_j = d_j src for the three axes; nb = number of 3D arrays.
// One derivative pass d_axis src -> dst over nb arrays.  FP64 arrays
// (SKY_KNOB_LINE_ARITH): 2 the digit-split operator on the tensor cores,
// 1 the FFT line pass in double-float arithmetic, 0 the FFT in FP64.
template <typename T>
static cudaError_t deriv_pass(Ctx* c, int ax, const cx<T>* src, cx<T>* dst, long long nb) {
  const int nx = c->n[0], ny = c->n[1], nz = c->n[2];
  const long long G = c->G;
  if constexpr (std::is_same<T, double>::value) {
    if (c->line_arith == 2 && c->d_dop[ax]) return deriv_tc(c, ax, src, dst, nb);
    if (c->line_arith >= 1) {
      OpDerivDD op{src, dst, c->d_ktdd[ax], G};
      auto go = [&](auto NC) -> cudaError_t {
        constexpr int N = decltype(NC)::value;
        if (ax == 0) return launch_line<dd, N, 0>(op, nx, ny, nz, nb, c);
        if (ax == 1) return launch_line<dd, N, 1>(op, nx, ny, nz, nb, c);
        return launch_line<dd, N, 2>(op, nx, ny, nz, nb, c);
      };
      return dispatch_n<false>(c->n[ax], go);
    }
  }
  OpDeriv<T> op{src, dst, kt_of<T>(c, ax), (T)(1.0 / c->n[ax]), G};
  auto go = [&](auto NC) -> cudaError_t {
    constexpr int N = decltype(NC)::value;
    if (ax == 0) return launch_line<T, N, 0>(op, nx, ny, nz, nb, c);
    if (ax == 1) return launch_line<T, N, 1>(op, nx, ny, nz, nb, c);
    return launch_line<T, N, 2>(op, nx, ny, nz, nb, c);
  };
  return dispatch_n<std::is_same<T, float>::value>(c->n[ax], go);
}

template <typename T>
static cudaError_t gradient_passes(Ctx* c, const cx<T>* src, cx<T>* const dst[3], long long nb) {
  for (int ax = 0; ax < 3; ++ax) {
    const cudaError_t e = deriv_pass<T>(c, ax, src, dst[ax], nb);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// ------------------------------------------------------------ apply_h kernels
// Spin-orbit matrices A_j = (sigma x W)_j acting on a spinor (v0, v1):
//   A_x v = (-Wy v0 - i Wz v1,  i Wz v0 + Wy v1)
//   A_y v = ( Wx v0 -   Wz v1,   -Wz v0 - Wx v1)
//   A_z v = ((Wy + i Wx) v1,    (Wy - i Wx) v0)
template <typename T>
__device__ __forceinline__ void apply_A(int j, T wx, T wy, T wz, cx<T> v0, cx<T> v1,
                                        cx<T>& o0, cx<T>& o1) {
  if (j == 0) {
    o0 = (-wy) * v0 + wz * mul_mi(v1);
    o1 = wz * mul_i(v0) + wy * v1;
  } else if (j == 1) {
    o0 = wx * v0 - wz * v1;
    o1 = (-wz) * v0 - wx * v1;
  } else {
    o0 = wy * v1 + wx * mul_i(v1);
    o1 = wy * v0 + wx * mul_mi(v0);
  }
}

// Pass 2: L -> hpsi, F_j -> G_j (in place).  grid.y = state within chunk.
template <typename T>
__global__ void __launch_bounds__(256) k_h_local(const cx<T>* __restrict__ psi, cx<T>* g0,
                                                 cx<T>* g1, cx<T>* g2, cx<T>* __restrict__ hpsi,
                                                 const double* __restrict__ U,
                                                 const double* __restrict__ B,
                                                 const double* __restrict__ W, int G) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= G) return;
  const long long o0 = (long long)blockIdx.y * 2 * G + p, o1 = o0 + G;
  const cx<T> a0 = psi[o0], a1 = psi[o1];
  const T u = (T)U[p], bb = (T)B[p];
  const T wx = (T)W[p], wy = (T)W[G + p], wz = (T)W[2 * G + p];
  cx<T>* gs[3] = {g0, g1, g2};
  cx<T> L0 = u * a0, L1 = u * a1;
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const cx<T> d0 = gs[j][o0], d1 = gs[j][o1];
    cx<T> t0, t1;
    apply_A<T>(j, wx, wy, wz, d0, d1, t0, t1);     // A_j G_j
    L0 = L0 + (T)0.5 * mul_mi(t0);                  // - (i/2) A_j G_j
    L1 = L1 + (T)0.5 * mul_mi(t1);
    apply_A<T>(j, wx, wy, wz, a0, a1, t0, t1);     // A_j psi
    gs[j][o0] = (-bb) * d0 + (T)0.5 * mul_mi(t0);   // F_j = -B G_j - (i/2) A_j psi
    gs[j][o1] = (-bb) * d1 + (T)0.5 * mul_mi(t1);
  }
  hpsi[o0] = L0;
  hpsi[o1] = L1;
}

// The same pass for the FP64 form in double-float arithmetic (the FP32 pipe;
// loads split, stores rounded by integer operations, dd.cuh).
__global__ void __launch_bounds__(256) k_h_local_dd(const double2* __restrict__ psi, double2* g0,
                                                    double2* g1, double2* g2,
                                                    double2* __restrict__ hpsi,
                                                    const double* __restrict__ U,
                                                    const double* __restrict__ B,
                                                    const double* __restrict__ W, int G) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= G) return;
  const long long o0 = (long long)blockIdx.y * 2 * G + p, o1 = o0 + G;
  const ddc a0 = ddc_of(psi[o0]), a1 = ddc_of(psi[o1]);
  const dd u = dd_of(U[p]), bb = dd_of(B[p]);
  const dd wx = dd_of(W[p]), wy = dd_of(W[G + p]), wz = dd_of(W[2 * G + p]);
  double2* gs[3] = {g0, g1, g2};
  ddc L0 = u * a0, L1 = u * a1;
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const ddc d0 = ddc_of(gs[j][o0]), d1 = ddc_of(gs[j][o1]);
    ddc t0, t1;
    apply_A<dd>(j, wx, wy, wz, d0, d1, t0, t1);    // A_j G_j
    L0 = L0 + half(mul_mi(t0));                    // - (i/2) A_j G_j
    L1 = L1 + half(mul_mi(t1));
    apply_A<dd>(j, wx, wy, wz, a0, a1, t0, t1);    // A_j psi
    gs[j][o0] = dbl2_of((-bb) * d0 + half(mul_mi(t0)));   // F_j = -B G_j - (i/2) A_j psi
    gs[j][o1] = dbl2_of((-bb) * d1 + half(mul_mi(t1)));
  }
  hpsi[o0] = dbl2_of(L0);
  hpsi[o1] = dbl2_of(L1);
}

// Deterministic block sum of two doubles (blockDim.x == kRedBlock).
__device__ __forceinline__ void block_sum2(double& a, double& b) {
  __shared__ double sa[kRedBlock / 32], sb[kRedBlock / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) { sa[w] = a; sb[w] = b; }
  __syncthreads();
  if (w == 0) {
    a = (l < kRedBlock / 32) ? sa[l] : 0.0;
    b = (l < kRedBlock / 32) ? sb[l] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_down_sync(0xffffffffu, a, o);
      b += __shfl_down_sync(0xffffffffu, b, o);
    }
  }
}

// Pass 4: hpsi = L + F_x + F_y + F_z; partial <psi|h psi>, |h psi|^2.
template <typename T>
__global__ void __launch_bounds__(kRedBlock) k_h_sum(const cx<T>* __restrict__ psi,
                                                     const cx<T>* __restrict__ g0,
                                                     const cx<T>* __restrict__ g1,
                                                     const cx<T>* __restrict__ g2,
                                                     cx<T>* __restrict__ hpsi, int G,
                                                     double* part, int nblk, int state0) {
  const long long base = (long long)blockIdx.y * 2 * G;
  double e = 0.0, n2 = 0.0;
  if constexpr (std::is_same<T, float>::value) {
    // FP32 arrays: exact products summed in float pairs (AccF), FP32 pipe
    AccF ae, an;
    for (int p = blockIdx.x * kRedBlock + threadIdx.x; p < 2 * G; p += nblk * kRedBlock) {
      const long long o = base + p;
      const cx<T> h = hpsi[o] + g0[o] + g1[o] + g2[o];
      hpsi[o] = h;
      const cx<T> ps = psi[o];
      ae.add_prod(ps.x, h.x);
      ae.add_prod(ps.y, h.y);
      an.add_prod(h.x, h.x);
      an.add_prod(h.y, h.y);
    }
    e = ae.value();
    n2 = an.value();
  } else {
    for (int p = blockIdx.x * kRedBlock + threadIdx.x; p < 2 * G; p += nblk * kRedBlock) {
      const long long o = base + p;
      const cx<T> h = hpsi[o] + g0[o] + g1[o] + g2[o];
      hpsi[o] = h;
      const double2 hd = to_d2(h), pd = to_d2(psi[o]);
      e += pd.x * hd.x + pd.y * hd.y;
      n2 += hd.x * hd.x + hd.y * hd.y;
    }
  }
  block_sum2(e, n2);
  if (threadIdx.x == 0) {
    double* dst = part + ((long long)(state0 + blockIdx.y) * nblk + blockIdx.x) * 2;
    dst[0] = e;
    dst[1] = n2;
  }
}

// Per-state totals of the partial sums, times dV.
__global__ void k_state_totals(const double* part, int nblk, int I, double dV,
                               double* eps, double* hn2) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= I) return;
  double a = 0.0, b = 0.0;
  for (int k = 0; k < nblk; ++k) {
    a += part[((long long)s * nblk + k) * 2];
    b += part[((long long)s * nblk + k) * 2 + 1];
  }
  if (eps) eps[s] = dV * a;
  if (hn2) hn2[s] = dV * b;
}

// ------------------------------------------------------------ fused FP32 h psi
// For FP32 arrays with every axis length up to 32, one pass per axis j
// computes that axis's whole share of h psi for a line of both spin
// components of one state:
//   G = d_j psi (the line in registers: forward transform, x i(k + theta/L)/N,
//   inverse), then point by point L_j = -(i/2) A_j G and F_j = -B G - (i/2)
//   A_j psi (F in place of G), then D_j = d_j F_j, and h psi += L_j + D_j
//   (h psi = U psi + L_x + D_x in the first pass);
// the last pass also forms <psi|h psi> and |h psi|^2.  The sum of the three
// passes is the rearranged h psi of the general path (identical terms, other
// rounding order), with h psi read and written once per pass and psi read
// once, instead of the gradient, local and divergence passes that write and
// re-read three scratch arrays.  States go in chunks whose psi and h psi stay
// in L2 across the passes.  Fields as floats (one conversion per call).
constexpr int kHaxLinesX = 32;      // lines per block along x (staged in shared memory)
constexpr int kHaxMaxN = 32;        // longest axis of the fused path
constexpr double kHaxL2Bytes = 48.0 * 1024 * 1024;   // psi + h psi of one chunk

struct HFields {
  const float* u;
  const float* b;
  const float* w;   // wx, wy, wz at w, w + G, w + 2 G
};

__global__ void k_fields_f32(const double* __restrict__ U, const double* __restrict__ B,
                             const double* __restrict__ W, int G, float* out) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= G) return;
  out[p] = (float)U[p];
  out[G + p] = (float)B[p];
  out[2 * G + p] = (float)W[p];
  out[3 * G + p] = (float)W[G + p];
  out[4 * G + p] = (float)W[2 * G + p];
}

// d_j of a line in place: forward transform, x i k_m / N, inverse.
template <int N>
__device__ __forceinline__ void deriv_line(float2 (&v)[N], const float* __restrict__ kt,
                                           float inv_n) {
  Fft<float, N, false>::run(v);
#pragma unroll
  for (int m = 0; m < N; ++m) {
    const float kk = __ldg(kt + m) * inv_n;
    v[m] = make_float2(-kk * v[m].y, kk * v[m].x);
  }
  Fft<float, N, true>::run(v);
}

// Point idx of the line: a = psi (both components), g = d_j psi -> F_j;
// returns L_j = -(i/2) A_j G in l0, l1.
template <int AXIS>
__device__ __forceinline__ void h_point(const HFields& f, int G, int idx, float2 a0, float2 a1,
                                        float2& g0, float2& g1, float2& l0, float2& l1) {
  const float bb = __ldg(f.b + idx);
  const float wx = __ldg(f.w + idx), wy = __ldg(f.w + G + idx), wz = __ldg(f.w + 2 * G + idx);
  float2 t0, t1;
  apply_A<float>(AXIS, wx, wy, wz, g0, g1, t0, t1);     // A_j G_j
  l0 = 0.5f * mul_mi(t0);
  l1 = 0.5f * mul_mi(t1);
  apply_A<float>(AXIS, wx, wy, wz, a0, a1, t0, t1);     // A_j psi
  g0 = (-bb) * g0 + 0.5f * mul_mi(t0);                  // F_j = -B G_j - (i/2) A_j psi
  g1 = (-bb) * g1 + 0.5f * mul_mi(t1);
}

// x pass (first): h psi = U psi + L_x + D_x.  A block stages nl <= kHaxLinesX
// consecutive x lines of both components of state blockIdx.y through shared
// memory (coalesced loads and stores; rows padded to N + 1).  One component's
// line at a time is transformed in registers; G, then F, of both components
// wait in gs[m][c][thread].
template <int N>
__global__ void __launch_bounds__(kHaxLinesX) k_h_axis_x(const float2* __restrict__ psi,
                                                         float2* __restrict__ hpsi, HFields f,
                                                         const float* __restrict__ kt,
                                                         float inv_n, int G, int rows) {
  __shared__ float2 tile[2][kHaxLinesX][N + 1];
  __shared__ float2 gs[N][2][kHaxLinesX];
  const int l0 = blockIdx.x * kHaxLinesX;
  const int nl = rows - l0 < kHaxLinesX ? rows - l0 : kHaxLinesX;
  const long long sb = (long long)blockIdx.y * 2 * G;
  const int tid = threadIdx.x;
  for (int e = tid; e < 2 * nl * N; e += kHaxLinesX) {
    const int c = e / (nl * N), r = e - c * nl * N;
    const int ll = r / N, m = r - ll * N;
    tile[c][ll][m] = psi[sb + (long long)c * G + (long long)(l0 + ll) * N + m];
  }
  __syncthreads();
  if (tid < nl) {
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      float2 v[N];
#pragma unroll
      for (int m = 0; m < N; ++m) v[m] = tile[c][tid][m];
      deriv_line<N>(v, kt, inv_n);
#pragma unroll
      for (int m = 0; m < N; ++m) gs[m][c][tid] = v[m];
    }
    const int base = (l0 + tid) * N;
#pragma unroll 4
    for (int m = 0; m < N; ++m) {
      const float2 a0 = tile[0][tid][m], a1 = tile[1][tid][m];
      float2 g0 = gs[m][0][tid], g1 = gs[m][1][tid], L0, L1;
      h_point<0>(f, G, base + m, a0, a1, g0, g1, L0, L1);
      gs[m][0][tid] = g0;
      gs[m][1][tid] = g1;
      const float u = __ldg(f.u + base + m);
      tile[0][tid][m] = u * a0 + L0;
      tile[1][tid][m] = u * a1 + L1;
    }
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      float2 v[N];
#pragma unroll
      for (int m = 0; m < N; ++m) v[m] = gs[m][c][tid];
      deriv_line<N>(v, kt, inv_n);
#pragma unroll
      for (int m = 0; m < N; ++m) tile[c][tid][m] = tile[c][tid][m] + v[m];
    }
  }
  __syncthreads();
  for (int e = tid; e < 2 * nl * N; e += kHaxLinesX) {
    const int c = e / (nl * N), r = e - c * nl * N;
    const int ll = r / N, m = r - ll * N;
    hpsi[sb + (long long)c * G + (long long)(l0 + ll) * N + m] = tile[c][ll][m];
  }
}

// Threads (lines) per block of the y / z pass: two shared arrays of N x 2
// values per thread (32 KiB at most).
__host__ __device__ constexpr int hax_threads(int N) { return N <= 16 ? 64 : 32; }

// y (AXIS 1) or z (AXIS 2) pass: one thread per line (consecutive threads on
// consecutive x: coalesced).  The line's G, then F, of both components wait in
// gs[m][c][thread] while one component's line is transformed in registers;
// L_j waits in ls.  Loads never follow a store to global memory within a
// phase (the pointwise phase stores to shared memory only; the last phase
// loads a component's old h psi values before storing any), so each thread's
// loads overlap instead of forming a chain of round trips.  The z pass (LAST)
// also adds this block's <psi|h psi> and |h psi|^2 (float-pair sums of exact
// products) to part[(state0 + state) * nblk + block].
template <int N, int AXIS, bool LAST>
__global__ void __launch_bounds__(hax_threads(N)) k_h_axis_yz(const float2* __restrict__ psi,
                                                              float2* __restrict__ hpsi,
                                                              HFields f,
                                                              const float* __restrict__ kt,
                                                              float inv_n, int nx, int ny, int G,
                                                              int lines, double* part, int nblk,
                                                              int state0) {
  constexpr int T = hax_threads(N);
  __shared__ float2 gs[N][2][T];
  __shared__ float2 ls[N][2][T];
  const int tid = threadIdx.x;
  const int l = blockIdx.x * T + tid;
  const long long sb = (long long)blockIdx.y * 2 * G;
  const float2* __restrict__ p0 = psi + sb;
  float2* __restrict__ h0 = hpsi + sb;
  const float* __restrict__ fb = f.b;
  const float* __restrict__ fw = f.w;
  AccF ae, an;
  if (l < lines) {
    const int x = l % nx, t = l / nx;
    const int base = AXIS == 1 ? t * ny * nx + x : t * nx + x;
    const int stride = AXIS == 1 ? nx : nx * ny;
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      float2 v[N];
#pragma unroll
      for (int m = 0; m < N; ++m) v[m] = p0[(long long)c * G + base + m * stride];
      deriv_line<N>(v, kt, inv_n);
#pragma unroll
      for (int m = 0; m < N; ++m) gs[m][c][tid] = v[m];
    }
#pragma unroll 8
    for (int m = 0; m < N; ++m) {
      const int idx = base + m * stride;
      const float2 a0 = p0[idx], a1 = p0[G + idx];
      const float bb = fb[idx];
      const float wx = fw[idx], wy = fw[G + idx], wz = fw[2 * G + idx];
      float2 g0 = gs[m][0][tid], g1 = gs[m][1][tid], t0, t1;
      apply_A<float>(AXIS, wx, wy, wz, g0, g1, t0, t1);     // A_j G_j
      ls[m][0][tid] = 0.5f * mul_mi(t0);                     // L_j = -(i/2) A_j G_j
      ls[m][1][tid] = 0.5f * mul_mi(t1);
      apply_A<float>(AXIS, wx, wy, wz, a0, a1, t0, t1);     // A_j psi
      gs[m][0][tid] = (-bb) * g0 + 0.5f * mul_mi(t0);       // F_j = -B G_j - (i/2) A_j psi
      gs[m][1][tid] = (-bb) * g1 + 0.5f * mul_mi(t1);
    }
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      float2 v[N];
#pragma unroll
      for (int m = 0; m < N; ++m) v[m] = gs[m][c][tid];
      deriv_line<N>(v, kt, inv_n);
      float2 hv[N];
#pragma unroll
      for (int m = 0; m < N; ++m) hv[m] = h0[(long long)c * G + base + m * stride];
#pragma unroll
      for (int m = 0; m < N; ++m) {
        v[m] = hv[m] + ls[m][c][tid] + v[m];
        h0[(long long)c * G + base + m * stride] = v[m];
      }
      if constexpr (LAST) {
#pragma unroll
        for (int m = 0; m < N; ++m) {
          const float2 a = p0[(long long)c * G + base + m * stride];
          ae.add_prod(a.x, v[m].x);
          ae.add_prod(a.y, v[m].y);
          an.add_prod(v[m].x, v[m].x);
          an.add_prod(v[m].y, v[m].y);
        }
      }
    }
  }
  if constexpr (LAST) {
    __shared__ double red[2][T / 32];
    double e = ae.value(), n2 = an.value();
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      e += __shfl_down_sync(0xffffffffu, e, o);
      n2 += __shfl_down_sync(0xffffffffu, n2, o);
    }
    if ((tid & 31) == 0) {
      red[0][tid >> 5] = e;
      red[1][tid >> 5] = n2;
    }
    __syncthreads();
    if (tid == 0) {
      double se = 0.0, sn = 0.0;
      for (int w = 0; w < T / 32; ++w) {
        se += red[0][w];
        sn += red[1][w];
      }
      double* dst = part + ((long long)(state0 + blockIdx.y) * nblk + blockIdx.x) * 2;
      dst[0] = se;
      dst[1] = sn;
    }
  }
}

bool fused_h_ok(const Ctx* c) {
  if (!c->d_hf) return false;
  if (c->prec == SKY_F64) return false;
  for (int j = 0; j < 3; ++j) {
    const int n = c->n[j];
    if (n != 8 && n != 12 && n != 16 && n != 20 && n != 24 && n != 32) return false;
  }
  return true;
}
int fused_h_blocks(const Ctx* c) {
  return (int)div_up((long long)c->n[0] * c->n[1], c->n[2] <= 16 ? 64 : 32);
}

// The three passes over states s0 .. s0 + ns - 1 (ps, hs: their arrays).
static cudaError_t fused_h_chunk(Ctx* c, const float2* ps, float2* hs, const HFields& f, int ns,
                                 int s0, int nblk) {
  const int nx = c->n[0], ny = c->n[1], nz = c->n[2], G = (int)c->G;
  cudaError_t e = dispatch_n<false>(nx, [&](auto Nc) -> cudaError_t {
    constexpr int N = decltype(Nc)::value;
    k_h_axis_x<N><<<dim3(div_up(ny * nz, kHaxLinesX), ns), kHaxLinesX, 0, c->stream>>>(
        ps, hs, f, c->d_ktf[0], 1.0f / nx, G, ny * nz);
    return cudaGetLastError();
  });
  if (e != cudaSuccess) return e;
  e = dispatch_n<false>(ny, [&](auto Nc) -> cudaError_t {
    constexpr int N = decltype(Nc)::value;
    constexpr int T = hax_threads(N);
    k_h_axis_yz<N, 1, false><<<dim3(div_up(nx * nz, T), ns), T, 0, c->stream>>>(
        ps, hs, f, c->d_ktf[1], 1.0f / ny, nx, ny, G, nx * nz, nullptr, 0, 0);
    return cudaGetLastError();
  });
  if (e != cudaSuccess) return e;
  e = dispatch_n<false>(nz, [&](auto Nc) -> cudaError_t {
    constexpr int N = decltype(Nc)::value;
    k_h_axis_yz<N, 2, true><<<dim3(nblk, ns), hax_threads(N), 0, c->stream>>>(
        ps, hs, f, c->d_ktf[2], 1.0f / nz, nx, ny, G, nx * ny, c->d_red, nblk, s0);
    return cudaGetLastError();
  });
  note_launch(3);
  return e;
}

static sky_status apply_h_fused(Ctx* c, const double* U, const double* B, const double* W,
                                const float2* psi, float2* hpsi, int I, double* eps, double* hn2) {
  const long long G = c->G, V = 2 * G;
  float* ff = c->d_hf;   // U, B, W as floats
  k_fields_f32<<<div_up(G, 256), 256, 0, c->stream>>>(U, B, W, (int)G, ff);
  note_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_check(c, e, "fused h psi fields");
  const HFields f{ff, ff + G, ff + 2 * G};
  const int nblk = fused_h_blocks(c);
  long long chunk = (long long)(kHaxL2Bytes / (2.0 * V * sizeof(float2)));
  if (chunk < 1) chunk = 1;
  for (int s0 = 0; s0 < I; s0 += (int)chunk) {
    const int ns = (I - s0) < chunk ? (I - s0) : (int)chunk;
    const float2* ps = psi + (long long)s0 * V;
    float2* hs = hpsi + (long long)s0 * V;
    e = fused_h_chunk(c, ps, hs, f, ns, s0, nblk);
    if (e != cudaSuccess) return cuda_check(c, e, "fused h psi");
  }
  if (eps || hn2) {
    k_state_totals<<<div_up(I, 128), 128, 0, c->stream>>>(c->d_red, nblk, I, c->dV, eps, hn2);
    note_launch();
    return cuda_check(c, cudaGetLastError(), "fused h psi totals");
  }
  return SKY_OK;
}

template <typename T>
static sky_status apply_h_t(Ctx* c, const double* U, const double* B, const double* W,
                            const cx<T>* psi, cx<T>* hpsi, int I, double* eps, double* hn2) {
  const long long G = c->G, V = 2 * G;
  cx<T>* scr = static_cast<cx<T>*>(c->d_gscr);
  const long long cstride = (long long)c->chunk * V;
  cx<T>* g[3] = {scr, scr + cstride, scr + 2 * cstride};
  for (int s0 = 0; s0 < I; s0 += c->chunk) {
    const int ns = (I - s0) < c->chunk ? (I - s0) : c->chunk;
    const cx<T>* ps = psi + (long long)s0 * V;
    cx<T>* hs = hpsi + (long long)s0 * V;
    cudaError_t e = gradient_passes<T>(c, ps, g, 2LL * ns);
    if (e != cudaSuccess) return cuda_check(c, e, "apply_h gradient");
    dim3 grid(div_up(G, 256), ns);
    if (std::is_same<T, double>::value && c->line_arith != 0)
      k_h_local_dd<<<grid, 256, 0, c->stream>>>((const double2*)ps, (double2*)g[0], (double2*)g[1],
                                                (double2*)g[2], (double2*)hs, U, B, W, (int)G);
    else
      k_h_local<T><<<grid, 256, 0, c->stream>>>(ps, g[0], g[1], g[2], hs, U, B, W, (int)G);
    note_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_check(c, e, "apply_h local");
    // pass 3: F_j <- d_j F_j in place, one axis per array
    for (int ax = 0; ax < 3; ++ax) {
      e = deriv_pass<T>(c, ax, g[ax], g[ax], 2LL * ns);
      if (e != cudaSuccess) return cuda_check(c, e, "apply_h divergence");
    }
    dim3 g4(c->red_nblk, ns);
    k_h_sum<T><<<g4, kRedBlock, 0, c->stream>>>(ps, g[0], g[1], g[2], hs, (int)G, c->d_red,
                                                c->red_nblk, s0); note_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_check(c, e, "apply_h sum");
  }
  if (eps || hn2) {
    k_state_totals<<<div_up(I, 128), 128, 0, c->stream>>>(c->d_red, c->red_nblk, I, c->dV,
                                                          eps, hn2); note_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_check(c, e, "apply_h totals");
  }
  return SKY_OK;
}

sky_status apply_h_impl(Ctx* c, const double* U, const double* B, const double* W,
                        const void* psi, void* hpsi, int I, double* eps, double* hn2) {
  if (c->prec == SKY_F64)
    return apply_h_t<double>(c, U, B, W, (const double2*)psi, (double2*)hpsi, I, eps, hn2);
  if (c->fused_h && fused_h_ok(c))
    return apply_h_fused(c, U, B, W, (const float2*)psi, (float2*)hpsi, I, eps, hn2);
  return apply_h_t<float>(c, U, B, W, (const float2*)psi, (float2*)hpsi, I, eps, hn2);
}

sky_status derivative_impl(Ctx* c, int axis, const void* src, void* dst, int n) {
  cudaError_t e;
  if (c->prec == SKY_F64)
    e = deriv_pass<double>(c, axis, (const double2*)src, (double2*)dst, n);
  else
    e = deriv_pass<float>(c, axis, (const float2*)src, (float2*)dst, n);
  return e == cudaSuccess ? SKY_OK : cuda_check(c, e, "derivative");
}

// ------------------------------------------------------------ damped step
__global__ void k_damp_table(double* P, const double* kx, const double* ky, const double* kz,
                             int nx, int ny, int nz, double hb2m, double E0) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= nx * ny * nz) return;
  const int x = p % nx, y = (p / nx) % ny, z = p / (nx * ny);
  const double k2 = kx[x] * kx[x] + ky[y] * ky[y] + kz[z] * kz[z];
  P[p] = 1.0 / (E0 + hb2m * k2);
}

template <typename T>
static sky_status damped_t(Ctx* c, int q, const cx<T>* psi, const cx<T>* hpsi,
                           const double* eps, cx<T>* phi, int I, double x0, double E0,
                           const float* w) {
  const int nx = c->n[0], ny = c->n[1], nz = c->n[2];
  const long long G = c->G;
  cudaError_t e;
  if (!(c->damp_E0[q] == E0)) {
    k_damp_table<<<div_up(G, 256), 256, 0, c->stream>>>(c->d_damp[q], c->d_kt[0], c->d_kt[1],
                                                        c->d_kt[2], nx, ny, nz, c->cp.hb2m[q], E0); note_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_check(c, e, "damping table");
    c->damp_E0[q] = E0;
  }
  if constexpr (std::is_same<T, double>::value) {
    if (c->line_arith == 2 && damp_tc_available(c)) {
      e = damp_tc(c, q, psi, hpsi, eps, phi, I, x0, w);
      return e == cudaSuccess ? SKY_OK : cuda_check(c, e, "damped step");
    }
  }
  const long long nb = 2LL * I;
  OpDampZFwd<T> o1{psi, hpsi, eps, phi, G};
  OpPass<T, false> o2{phi, G};
  OpDampX<T> o3{phi, c->d_damp[q], (T)(x0 / (double)G), G};
  OpPass<T, true> o4{phi, G};
  OpDampZInv<T> o5{psi, phi, w, G};
  constexpr bool L = std::is_same<T, float>::value;
  e = dispatch_n<L>(nz, [&](auto NC) { return launch_line<T, decltype(NC)::value, 2>(o1, nx, ny, nz, nb, c); });
  if (e == cudaSuccess)
    e = dispatch_n<L>(ny, [&](auto NC) { return launch_line<T, decltype(NC)::value, 1>(o2, nx, ny, nz, nb, c); });
  if (e == cudaSuccess)
    e = dispatch_n<L>(nx, [&](auto NC) { return launch_line<T, decltype(NC)::value, 0>(o3, nx, ny, nz, nb, c); });
  if (e == cudaSuccess)
    e = dispatch_n<L>(ny, [&](auto NC) { return launch_line<T, decltype(NC)::value, 1>(o4, nx, ny, nz, nb, c); });
  if (e == cudaSuccess)
    e = dispatch_n<L>(nz, [&](auto NC) { return launch_line<T, decltype(NC)::value, 2>(o5, nx, ny, nz, nb, c); });
  return e == cudaSuccess ? SKY_OK : cuda_check(c, e, "damped step");
}

sky_status damped_step_impl(Ctx* c, int q, const void* psi, const void* hpsi,
                            const double* eps, void* phi, int I, double x0, double E0,
                            const float* w) {
  if (c->prec == SKY_F64)
    return damped_t<double>(c, q, (const double2*)psi, (const double2*)hpsi, eps,
                            (double2*)phi, I, x0, E0, w);
  return damped_t<float>(c, q, (const float2*)psi, (const float2*)hpsi, eps, (float2*)phi, I,
                         x0, E0, w);
}

// ------------------------------------------------------------ densities
// Partial rho, tau, J over the states of one split:
//   M_kj = psi^+ sigma_k G_j, J_x = Im M_zy - Im M_yz, J_y = Im M_xz - Im M_zx,
//   J_z = Im M_yx - Im M_xy  (J_i = sum_jk eps_ijk Re[-i M_kj] = sum eps_ijk Im M_kj).
template <typename T>
__global__ void __launch_bounds__(128) k_dens_accum(const cx<T>* __restrict__ psi,
                                                    const cx<T>* __restrict__ g0,
                                                    const cx<T>* __restrict__ g1,
                                                    const cx<T>* __restrict__ g2, int G, int ns,
                                                    int per_split, double* part) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= G) return;
  const int s_beg = blockIdx.y * per_split;
  const int s_end = (s_beg + per_split) < ns ? (s_beg + per_split) : ns;
  double rho = 0, tau = 0, jx = 0, jy = 0, jz = 0;
  const cx<T>* gs[3] = {g0, g1, g2};
  if constexpr (std::is_same<T, float>::value) {
    // FP32 arrays: every product exact as a float pair, the sums in float
    // pairs (AccF) on the FP32 pipe; the same terms as the FP64 loop below,
    // with X(s, t, j) = conj(a_s) d_t along j:
    //   Im M_xj = Im X(0,1,j) + Im X(1,0,j), Im M_yj = Re X(1,0,j) - Re X(0,1,j),
    //   Im M_zj = Im X(0,0,j) - Im X(1,1,j)
    AccF r, ta, ax, ay, az;
    for (int s = s_beg; s < s_end; ++s) {
      const long long o0 = (long long)s * 2 * G + p, o1 = o0 + G;
      const float2 a0 = psi[o0], a1 = psi[o1];
      r.add_prod(a0.x, a0.x); r.add_prod(a0.y, a0.y);
      r.add_prod(a1.x, a1.x); r.add_prod(a1.y, a1.y);
      float2 d0[3], d1[3];
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        d0[j] = gs[j][o0];
        d1[j] = gs[j][o1];
        ta.add_prod(d0[j].x, d0[j].x); ta.add_prod(d0[j].y, d0[j].y);
        ta.add_prod(d1[j].x, d1[j].x); ta.add_prod(d1[j].y, d1[j].y);
      }
      // J_x = Im M_zy - Im M_yz
      ax.im_cj(1.0f, a0, d0[1]); ax.im_cj(-1.0f, a1, d1[1]);
      ax.re_cj(-1.0f, a1, d0[2]); ax.re_cj(1.0f, a0, d1[2]);
      // J_y = Im M_xz - Im M_zx
      ay.im_cj(1.0f, a0, d1[2]); ay.im_cj(1.0f, a1, d0[2]);
      ay.im_cj(-1.0f, a0, d0[0]); ay.im_cj(1.0f, a1, d1[0]);
      // J_z = Im M_yx - Im M_xy
      az.re_cj(1.0f, a1, d0[0]); az.re_cj(-1.0f, a0, d1[0]);
      az.im_cj(-1.0f, a0, d1[1]); az.im_cj(-1.0f, a1, d0[1]);
    }
    rho = r.value(); tau = ta.value(); jx = ax.value(); jy = ay.value(); jz = az.value();
  } else {
  for (int s = s_beg; s < s_end; ++s) {
    const long long o0 = (long long)s * 2 * G + p, o1 = o0 + G;
    const double2 a0 = to_d2(psi[o0]), a1 = to_d2(psi[o1]);
    rho += a0.x * a0.x + a0.y * a0.y + a1.x * a1.x + a1.y * a1.y;
    double imx[3], imy[3], imz[3];   // Im M_{x,j}, Im M_{y,j}, Im M_{z,j}
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const double2 d0 = to_d2(gs[j][o0]), d1 = to_d2(gs[j][o1]);
      tau += d0.x * d0.x + d0.y * d0.y + d1.x * d1.x + d1.y * d1.y;
      const double2 c01 = cmulc(a0, d1), c10 = cmulc(a1, d0);   // conj(a0) d1, conj(a1) d0
      const double2 c00 = cmulc(a0, d0), c11 = cmulc(a1, d1);
      imx[j] = c01.y + c10.y;
      imy[j] = c10.x - c01.x;
      imz[j] = c00.y - c11.y;
    }
    jx += imz[1] - imy[2];
    jy += imx[2] - imz[0];
    jz += imy[0] - imx[1];
  }
  }
  double* dst = part + (long long)blockIdx.y * 5 * G;
  dst[p] = rho;
  dst[G + p] = tau;
  dst[2 * G + p] = jx;
  dst[3 * G + p] = jy;
  dst[4 * G + p] = jz;
}

// Sum the splits in order; accumulate onto the outputs after the first chunk.
__global__ void k_dens_reduce(const double* part, int nsplit, int G, int accumulate,
                              double* rho, double* tau, double* J) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= G) return;
  double v[5] = {0, 0, 0, 0, 0};
  for (int s = 0; s < nsplit; ++s)
#pragma unroll
    for (int f = 0; f < 5; ++f) v[f] += part[((long long)s * 5 + f) * G + p];
  if (accumulate) {
    rho[p] += v[0]; tau[p] += v[1];
    J[p] += v[2]; J[G + p] += v[3]; J[2 * G + p] += v[4];
  } else {
    rho[p] = v[0]; tau[p] = v[1];
    J[p] = v[2]; J[G + p] = v[3]; J[2 * G + p] = v[4];
  }
}

sky_status field_divergence(Ctx* c, const double* J, double* divJ);  // fields.cu

template <typename T>
static sky_status densities_t(Ctx* c, const cx<T>* psi, int I, double* rho, double* tau,
                              double* J, double* divJ) {
  const long long G = c->G, V = 2 * G;
  cx<T>* scr = static_cast<cx<T>*>(c->d_gscr);
  const long long cstride = (long long)c->chunk * V;
  cx<T>* g[3] = {scr, scr + cstride, scr + 2 * cstride};
  double* Jout = J ? J : c->d_ftmp + 13 * G;   // [3][G] temporaries when J not wanted
  if (I == 0) {
    cudaMemsetAsync(rho, 0, G * sizeof(double), c->stream);
    cudaMemsetAsync(tau, 0, G * sizeof(double), c->stream);
    cudaMemsetAsync(Jout, 0, 3 * G * sizeof(double), c->stream);
  }
  for (int s0 = 0; s0 < I; s0 += c->chunk) {
    const int ns = (I - s0) < c->chunk ? (I - s0) : c->chunk;
    const cx<T>* ps = psi + (long long)s0 * V;
    cudaError_t e = gradient_passes<T>(c, ps, g, 2LL * ns);
    if (e != cudaSuccess) return cuda_check(c, e, "densities gradient");
    const int per = (ns + kDensSplits - 1) / kDensSplits;
    const int nsplit = (ns + per - 1) / per;
    dim3 grid(div_up(G, 128), nsplit);
    k_dens_accum<T><<<grid, 128, 0, c->stream>>>(ps, g[0], g[1], g[2], (int)G, ns, per, c->d_dpart); note_launch();
    k_dens_reduce<<<div_up(G, 256), 256, 0, c->stream>>>(c->d_dpart, nsplit, (int)G, s0 > 0, rho,
                                                         tau, Jout); note_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_check(c, e, "densities accumulate");
  }
  if (divJ) return field_divergence(c, Jout, divJ);
  return SKY_OK;
}

sky_status densities_impl(Ctx* c, const void* psi, int I, double* rho, double* tau, double* J,
                          double* divJ) {
  if (c->prec == SKY_F64)
    return densities_t<double>(c, (const double2*)psi, I, rho, tau, J, divJ);
  return densities_t<float>(c, (const float2*)psi, I, rho, tau, J, divJ);
}

}  // namespace sky
