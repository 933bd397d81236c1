// Register-resident mixed-radix FFTs along one axis of batched 3D arrays.
//
// Every derivative of the method is spectral (Sec. 2.2: "We use FFTs to
// compute the derivatives").  A derivative along axis j only needs the 1D
// transform along j: the transforms along the other two axes cancel, so
// d_j f = IFFT_j[ i k_j FFT_j[f] ] exactly.  One thread owns one line of N
// points in registers; the radix-4/2/3/5 decimation-in-time recursion is
// fully unrolled at compile time, so twiddle indices are constants and
// quarter-turn twiddles cost nothing.  Lines along y and z are read with
// consecutive threads on consecutive x (coalesced); lines along x are staged
// through shared memory (rows padded to N+1 to avoid bank conflicts).
#pragma once

#include "dd.cuh"

namespace sky {

// ------------------------------------------------------------ twiddles
// W_N^p tables (cos, sin of 2 pi p / N) for every transform length that
// appears at some level of the recursion.
constexpr int kNumTw = 11;
__host__ __device__ constexpr int tw_size(int i) {
  return i == 0 ? 6 : i == 1 ? 8 : i == 2 ? 10 : i == 3 ? 12 : i == 4 ? 16 : i == 5 ? 20
       : i == 6 ? 24 : i == 7 ? 32 : i == 8 ? 40 : i == 9 ? 48 : i == 10 ? 64 : 0;
}
__host__ __device__ constexpr int tw_offset(int N) {
  int off = 0;
  for (int i = 0; i < kNumTw; ++i) {
    if (tw_size(i) == N) return off;
    off += tw_size(i);
  }
  return -1;
}
constexpr int kTwTotal = 6 + 8 + 10 + 12 + 16 + 20 + 24 + 32 + 40 + 48 + 64;

// One copy per translation unit (no relocatable device code); each unit
// uploads its own copy for the current device at context creation.
static __constant__ double2 c_tw_d[kTwTotal];
static __constant__ float2 c_tw_f[kTwTotal];
static __constant__ float4 c_tw_dd[kTwTotal];   // (cos hi, cos lo, sin hi, sin lo)

static inline cudaError_t upload_twiddles_this_unit() {
  double2 hd[kTwTotal];
  float2 hf[kTwTotal];
  float4 hdd[kTwTotal];
  const long double two_pi = 6.283185307179586476925286766559005768L;
  for (int i = 0; i < kNumTw; ++i) {
    const int N = tw_size(i), off = tw_offset(N);
    for (int p = 0; p < N; ++p) {
      const long double a = two_pi * (long double)p / (long double)N;
      hd[off + p] = make_double2((double)cosl(a), (double)sinl(a));
      hf[off + p] = make_float2((float)cosl(a), (float)sinl(a));
      const float ch = (float)cosl(a), sh = (float)sinl(a);
      hdd[off + p] = make_float4(ch, (float)(cosl(a) - (long double)ch), sh,
                                 (float)(sinl(a) - (long double)sh));
    }
  }
  cudaError_t e = cudaMemcpyToSymbol(c_tw_d, hd, sizeof(hd));
  if (e != cudaSuccess) return e;
  e = cudaMemcpyToSymbol(c_tw_dd, hdd, sizeof(hdd));
  if (e != cudaSuccess) return e;
  return cudaMemcpyToSymbol(c_tw_f, hf, sizeof(hf));
}

template <typename T> __device__ __forceinline__ cx<T> tw_entry(int i);
template <> __device__ __forceinline__ double2 tw_entry<double>(int i) { return c_tw_d[i]; }
template <> __device__ __forceinline__ float2 tw_entry<float>(int i) { return c_tw_f[i]; }
template <> __device__ __forceinline__ ddc tw_entry<dd>(int i) {
  const float4 w = c_tw_dd[i];
  return ddc{dd(w.x, w.y), dd(w.z, w.w)};
}

// v * W_N^p with W_N = exp(-2 pi i / N) (forward) or exp(+2 pi i / N) (inverse).
template <typename T, int N, bool INV>
__device__ __forceinline__ cx<T> twiddle(int p, cx<T> v) {
  if (p == 0) return v;
  if ((4 * p) % N == 0) {
    const int q = (4 * p) / N;
    if (q == 2) return -v;
    return ((q == 1) != INV) ? mul_mi(v) : mul_i(v);
  }
  const cx<T> w = tw_entry<T>(tw_offset(N) + p);
  const T c = w.x, s = INV ? w.y : -w.y;
  return mkc<T>(v.x * c - v.y * s, v.x * s + v.y * c);
}

// ------------------------------------------------------------ small DFTs
template <typename T, int R, bool INV> struct Dft;

template <typename T, bool INV> struct Dft<T, 1, INV> {
  static __device__ __forceinline__ void run(cx<T>*) {}
};
template <typename T, bool INV> struct Dft<T, 2, INV> {
  static __device__ __forceinline__ void run(cx<T>* x) {
    const cx<T> a = x[0], b = x[1];
    x[0] = a + b; x[1] = a - b;
  }
};
template <typename T, bool INV> struct Dft<T, 4, INV> {
  static __device__ __forceinline__ void run(cx<T>* x) {
    const cx<T> a = x[0] + x[2], b = x[0] - x[2], c = x[1] + x[3], d = x[1] - x[3];
    x[0] = a + c; x[2] = a - c;
    x[1] = INV ? b + mul_i(d) : b + mul_mi(d);
    x[3] = INV ? b + mul_mi(d) : b + mul_i(d);
  }
};
template <typename T, bool INV> struct Dft<T, 3, INV> {
  // X1,2 = x0 - (x1+x2)/2 -/+ i (sqrt3/2)(x1 - x2) for the forward sign.
  static __device__ __forceinline__ void run(cx<T>* x) {
    constexpr T h = T(0.866025403784438646763723170752936183);
    constexpr T half = T(0.5);
    const cx<T> s = x[1] + x[2], d = x[1] - x[2];
    const cx<T> m = x[0] - half * s;
    const cx<T> r = h * (INV ? mul_i(d) : mul_mi(d));
    x[0] = x[0] + s; x[1] = m + r; x[2] = m - r;
  }
};
template <typename T, bool INV> struct Dft<T, 5, INV> {
  // c1 = cos(2pi/5), c2 = cos(4pi/5), s1 = sin(2pi/5), s2 = sin(4pi/5).
  static __device__ __forceinline__ void run(cx<T>* x) {
    constexpr T c1 = T(0.309016994374947424102293417182819059);
    constexpr T c2 = T(-0.809016994374947424102293417182819059);
    constexpr T s1 = T(0.951056516295153572116439333379382143);
    constexpr T s2 = T(0.587785252292473129181428776797681326);
    const cx<T> a1 = x[1] + x[4], a2 = x[2] + x[3], b1 = x[1] - x[4], b2 = x[2] - x[3];
    const cx<T> m1 = x[0] + c1 * a1 + c2 * a2, m2 = x[0] + c2 * a1 + c1 * a2;
    const cx<T> n1 = s1 * b1 + s2 * b2, n2 = s2 * b1 - s1 * b2;
    const cx<T> r1 = INV ? mul_i(n1) : mul_mi(n1), r2 = INV ? mul_i(n2) : mul_mi(n2);
    x[0] = x[0] + a1 + a2;
    x[1] = m1 + r1; x[4] = m1 - r1;
    x[2] = m2 + r2; x[3] = m2 - r2;
  }
};

__host__ __device__ constexpr int radix_of(int N) {
  return (N <= 5 && N != 4) ? N : (N == 4 ? 4 : (N % 4 == 0 ? 4 : (N % 2 == 0 ? 2 : -1)));
}

// Unnormalised DFT of length N in registers, X_k = sum_n x_n W_N^{nk}.
// N = R*M: n = r + R m, k = k1 + M k2;  X = sum_r W_R^{r k2} W_N^{r k1} Y_r[k1].
template <typename T, int N, bool INV> struct Fft {
  static constexpr int R = radix_of(N);
  static constexpr int M = N / R;
  static_assert(R > 0, "unsupported transform length");
  static __device__ __forceinline__ void run(cx<T>* x) {
    if constexpr (M == 1) {
      Dft<T, N, INV>::run(x);
    } else {
      cx<T> y[N];
#pragma unroll
      for (int r = 0; r < R; ++r)
#pragma unroll
        for (int m = 0; m < M; ++m) y[r * M + m] = x[r + R * m];
#pragma unroll
      for (int r = 0; r < R; ++r) Fft<T, M, INV>::run(y + r * M);
#pragma unroll
      for (int k1 = 0; k1 < M; ++k1) {
        cx<T> t[R];
#pragma unroll
        for (int r = 0; r < R; ++r) t[r] = twiddle<T, N, INV>(r * k1, y[r * M + k1]);
        Dft<T, R, INV>::run(t);
#pragma unroll
        for (int k2 = 0; k2 < R; ++k2) x[k1 + M * k2] = t[k2];
      }
    }
  }
};

// ------------------------------------------------------------ line passes
// Geometry of one pass: `nbatch` 3D arrays of nx*ny*nz points, batch stride G.
struct LineGeom {
  int nx, ny, nz;
  long long nlines;   // nbatch * G / N
};

constexpr int kLineThreads = 128;   // most threads (= lines) per block along y, z
constexpr int kLinesX = 64;         // most lines per block along x (smem staged)
// The block shapes actually launched come from the context (tunable):
// Ctx::line_yz in {32, 64, 128}, Ctx::line_x in {16, 32, 64}.

// An Op provides:
//   static constexpr bool kFwd, kInv;
//   cx<T> load(long long b, int idx) const;          element idx of array b
//   void mid(cx<T>& v, long long b, int idx, int m) const;   after forward
//   void store(long long b, int idx, cx<T> v) const;
// idx is the point index within one array, m the position along the line.
template <typename T, int N, class Op>
__device__ __forceinline__ void process_line(const Op& op, cx<T>* v, long long b, int base,
                                             int stride) {
  if constexpr (Op::kFwd) Fft<T, N, false>::run(v);
#pragma unroll
  for (int m = 0; m < N; ++m) op.mid(v[m], b, base + m * stride, m);
  if constexpr (Op::kInv) Fft<T, N, true>::run(v);
}

// Lines along y (AXIS = 1) or z (AXIS = 2): one thread per line, direct loads.
template <typename T, int N, int AXIS, class Op>
__global__ void __launch_bounds__(kLineThreads) k_line_yz(Op op, LineGeom g) {
  const long long l = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= g.nlines) return;
  const int x = (int)(l % g.nx);
  const long long t = l / g.nx;
  long long b;
  int base, stride;
  if constexpr (AXIS == 1) {
    const int z = (int)(t % g.nz);
    b = t / g.nz;
    base = z * g.ny * g.nx + x;
    stride = g.nx;
  } else {
    const int y = (int)(t % g.ny);
    b = t / g.ny;
    base = y * g.nx + x;
    stride = g.nx * g.ny;
  }
  cx<T> v[N];
#pragma unroll
  for (int m = 0; m < N; ++m) v[m] = op.load(b, base + m * stride);
  process_line<T, N>(op, v, b, base, stride);
#pragma unroll
  for (int m = 0; m < N; ++m) op.store(b, base + m * stride, v[m]);
}

// Lines along x: a block stages blockDim.x (<= kLinesX) contiguous lines
// through shared memory.
template <typename T, int N, class Op>
__global__ void __launch_bounds__(kLinesX) k_line_x(Op op, LineGeom g) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* tile = reinterpret_cast<cx<T>*>(smem_raw);   // [lx][N + 1]
  __shared__ long long s_b[kLinesX];
  __shared__ int s_r[kLinesX];
  const int lx = blockDim.x;
  const long long l0 = (long long)blockIdx.x * lx;
  const int rows = g.ny * g.nz;
  const int nl = (int)((g.nlines - l0) < lx ? (g.nlines - l0) : lx);
  if ((int)threadIdx.x < nl) {
    const long long l = l0 + threadIdx.x;
    s_b[threadIdx.x] = l / rows;
    s_r[threadIdx.x] = (int)(l % rows);
  }
  __syncthreads();
  for (int e = threadIdx.x; e < nl * N; e += lx) {
    const int ll = e / N, m = e % N;
    tile[ll * (N + 1) + m] = op.load(s_b[ll], s_r[ll] * N + m);
  }
  __syncthreads();
  if ((int)threadIdx.x < nl) {
    const int ll = threadIdx.x;
    cx<T> v[N];
#pragma unroll
    for (int m = 0; m < N; ++m) v[m] = tile[ll * (N + 1) + m];
    process_line<T, N>(op, v, s_b[ll], s_r[ll] * N, 1);
#pragma unroll
    for (int m = 0; m < N; ++m) tile[ll * (N + 1) + m] = v[m];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < nl * N; e += lx) {
    const int ll = e / N, m = e % N;
    op.store(s_b[ll], s_r[ll] * N + m, tile[ll * (N + 1) + m]);
  }
}

// Launch one pass along `axis` over `nbatch` arrays on the context's stream,
// with the context's block shapes.
template <typename T, int N, int AXIS, class Op>
inline cudaError_t launch_line(const Op& op, int nx, int ny, int nz, long long nbatch,
                               const Ctx* c) {
  LineGeom g;
  g.nx = nx; g.ny = ny; g.nz = nz;
  const long long G = (long long)nx * ny * nz;
  g.nlines = nbatch * (G / N);
  if (g.nlines == 0) return cudaSuccess;
  if constexpr (AXIS == 0) {
    const int lx = c->line_x;
    const size_t smem = (size_t)lx * (N + 1) * sizeof(cx<T>);
    constexpr size_t kSmemMax = (size_t)kLinesX * (N + 1) * sizeof(cx<T>);
    if constexpr (kSmemMax > 48 * 1024) {
      // opt in above 48 KB once per device (before any stream capture)
      static bool opted[64] = {false};
      int dev = 0;
      cudaError_t e = cudaGetDevice(&dev);
      if (e != cudaSuccess) return e;
      if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
      if (!opted[dev]) {
        e = cudaFuncSetAttribute(k_line_x<T, N, Op>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kSmemMax);
        if (e != cudaSuccess) return e;
        opted[dev] = true;
      }
    }
    k_line_x<T, N, Op><<<div_up(g.nlines, lx), lx, smem, c->stream>>>(op, g); note_launch();
  } else {
    const int ly = c->line_yz;
    k_line_yz<T, N, AXIS, Op><<<div_up(g.nlines, ly), ly, 0, c->stream>>>(op, g); note_launch();
  }
  return cudaGetLastError();
}

// Run f(std::integral_constant<int, N>) for the runtime axis length n.
template <bool WITH_LARGE, typename F>
inline cudaError_t dispatch_n(int n, F&& f) {
  switch (n) {
    case 8: return f(std::integral_constant<int, 8>{});
    case 12: return f(std::integral_constant<int, 12>{});
    case 16: return f(std::integral_constant<int, 16>{});
    case 20: return f(std::integral_constant<int, 20>{});
    case 24: return f(std::integral_constant<int, 24>{});
    case 32: return f(std::integral_constant<int, 32>{});
    case 48: if constexpr (WITH_LARGE) return f(std::integral_constant<int, 48>{}); break;
    case 64: if constexpr (WITH_LARGE) return f(std::integral_constant<int, 64>{}); break;
    default: break;
  }
  return cudaErrorInvalidValue;
}

}  // namespace sky
