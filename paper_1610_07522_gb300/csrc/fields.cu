// Mean fields, Coulomb potential, energy and the convergence measure
// (Eq. Skyrme, Sec. 2.2, Eq. convergence).  Fields are FP64 for every
// spinor precision; real-field derivatives are spectral with the plain
// wavenumbers, real part kept.
#include "fft_lines.cuh"

namespace sky {

sky_status upload_twiddles_fields(Ctx* c) {
  return cuda_check(c, upload_twiddles_this_unit(), "twiddle upload (fields)");
}

// out (= or +=) Re IFFT[ mult FFT[in] ] along one axis; mult = i k (mode 0)
// or -k^2 (mode 1), divided by N.
struct OpRealD {
  static constexpr bool kFwd = true, kInv = true;
  const double* in; double* out; const double* k; double inv_n; int mode; int acc; long long G;
  __device__ __forceinline__ double2 load(long long b, int i) const {
    return make_double2(in[b * G + i], 0.0);
  }
  __device__ __forceinline__ void mid(double2& v, long long, int, int m) const {
    if (mode == 0) {
      const double kk = k[m] * inv_n;
      v = make_double2(-kk * v.y, kk * v.x);
    } else {
      const double f = -k[m] * k[m] * inv_n;
      v = make_double2(f * v.x, f * v.y);
    }
  }
  __device__ __forceinline__ void store(long long b, int i, double2 v) const {
    out[b * G + i] = acc ? out[b * G + i] + v.x : v.x;
  }
};

struct OpR2CFwd {   // real in -> complex, forward
  static constexpr bool kFwd = true, kInv = false;
  const double* in; double2* out; long long G;
  __device__ __forceinline__ double2 load(long long b, int i) const { return make_double2(in[b * G + i], 0.0); }
  __device__ __forceinline__ void mid(double2&, long long, int, int) const {}
  __device__ __forceinline__ void store(long long b, int i, double2 v) const { out[b * G + i] = v; }
};
template <bool INV> struct OpCPass {
  static constexpr bool kFwd = !INV, kInv = INV;
  double2* a; long long G;
  __device__ __forceinline__ double2 load(long long b, int i) const { return a[b * G + i]; }
  __device__ __forceinline__ void mid(double2&, long long, int, int) const {}
  __device__ __forceinline__ void store(long long b, int i, double2 v) const { a[b * G + i] = v; }
};
struct OpCoulX {    // forward x, times 4 pi e^2 / (G |k|^2), inverse x
  static constexpr bool kFwd = true, kInv = true;
  double2* a; const double* Pc; double scale; long long G;
  __device__ __forceinline__ double2 load(long long b, int i) const { return a[b * G + i]; }
  __device__ __forceinline__ void mid(double2& v, long long, int i, int) const {
    const double f = Pc[i] * scale;
    v = make_double2(f * v.x, f * v.y);
  }
  __device__ __forceinline__ void store(long long b, int i, double2 v) const { a[b * G + i] = v; }
};
struct OpC2RInv {   // inverse z, real part out
  static constexpr bool kFwd = false, kInv = true;
  const double2* a; double* out; long long G;
  __device__ __forceinline__ double2 load(long long b, int i) const { return a[b * G + i]; }
  __device__ __forceinline__ void mid(double2&, long long, int, int) const {}
  __device__ __forceinline__ void store(long long b, int i, double2 v) const { out[b * G + i] = v.x; }
};

template <class Op>
static cudaError_t run_pass(Ctx* c, int axis, const Op& op, long long nb) {
  const int nx = c->n[0], ny = c->n[1], nz = c->n[2];
  return dispatch_n<true>(c->n[axis], [&](auto NC) -> cudaError_t {
    constexpr int N = decltype(NC)::value;
    if (axis == 0) return launch_line<double, N, 0>(op, nx, ny, nz, nb, c);
    if (axis == 1) return launch_line<double, N, 1>(op, nx, ny, nz, nb, c);
    return launch_line<double, N, 2>(op, nx, ny, nz, nb, c);
  });
}

// out = sum_axis (derivative or second derivative) of nb fields.
static cudaError_t real_op_sum(Ctx* c, const double* in, double* out, long long nb, int mode) {
  for (int ax = 0; ax < 3; ++ax) {
    OpRealD op{in, out, c->d_kp[ax], 1.0 / c->n[ax], mode, ax > 0, (long long)c->G};
    cudaError_t e = run_pass(c, ax, op, nb);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// divJ = sum_i d_i J_i for one [3][G] vector field.
sky_status field_divergence(Ctx* c, const double* J, double* divJ) {
  const long long G = c->G;
  for (int ax = 0; ax < 3; ++ax) {
    OpRealD op{J + ax * G, divJ, c->d_kp[ax], 1.0 / c->n[ax], 0, ax > 0, G};
    cudaError_t e = run_pass(c, ax, op, 1);
    if (e != cudaSuccess)
      return set_err(c, SKY_ECUDA, "divergence (axis %d, n %d, blocks %d/%d): %s", ax, c->n[ax],
                     c->line_x, c->line_yz, cudaGetErrorString(e));
  }
  return SKY_OK;
}

// Temporaries in d_ftmp ([16][G]): 0-1 rho_T, 2-3 Delta rho_T,
// 4-9 d_j rho_T at 4 + 2j + T, 10 V_C, 11-12 reduction partials,
// 13-15 spin-orbit density when the caller does not want it.
__global__ void k_isospin(const double* rho, double* rT, int G) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= G) return;
  rT[p] = rho[p] + rho[G + p];
  rT[G + p] = rho[p] - rho[G + p];
}

__global__ void k_coul_table(double* Pc, const double* kx, const double* ky, const double* kz,
                             int nx, int ny, int nz, double e2) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= nx * ny * nz) return;
  const int x = p % nx, y = (p / nx) % ny, z = p / (nx * ny);
  const double k2 = kx[x] * kx[x] + ky[y] * ky[y] + kz[z] * kz[z];
  Pc[p] = k2 > 0.0 ? 4.0 * 3.14159265358979323846 * e2 / k2 : 0.0;
}

sky_status build_coulomb_table(Ctx* c) {
  k_coul_table<<<div_up(c->G, 256), 256, 0, c->stream>>>(c->d_coul, c->d_kp[0], c->d_kp[1],
                                                         c->d_kp[2], c->n[0], c->n[1], c->n[2],
                                                         c->cp.e2); note_launch();
  return cuda_check(c, cudaGetLastError(), "coulomb table");
}

// Shared first part of mean fields and energy: rho_T, Delta rho_T, grad rho_T, V_C.
static sky_status field_prep(Ctx* c, const double* rho, bool need_grad) {
  const long long G = c->G;
  double* f = c->d_ftmp;
  cudaError_t e;
  k_isospin<<<div_up(G, 256), 256, 0, c->stream>>>(rho, f, (int)G); note_launch();
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_check(c, e, "isospin");
  if ((e = real_op_sum(c, f, f + 2 * G, 2, 1)) != cudaSuccess) return cuda_check(c, e, "laplacian");
  if (need_grad) {
    for (int ax = 0; ax < 3; ++ax) {
      OpRealD op{f, f + (4 + 2 * ax) * G, c->d_kp[ax], 1.0 / c->n[ax], 0, 0, G};
      if ((e = run_pass(c, ax, op, 2)) != cudaSuccess) return cuda_check(c, e, "gradient");
    }
  }
  if (c->cp.coulomb) {
    OpR2CFwd o1{rho + G, c->d_fcx, G};
    OpCPass<false> o2{c->d_fcx, G};
    OpCoulX o3{c->d_fcx, c->d_coul, 1.0 / (double)G, G};
    OpCPass<true> o4{c->d_fcx, G};
    OpC2RInv o5{c->d_fcx, f + 10 * G, G};
    if ((e = run_pass(c, 2, o1, 1)) == cudaSuccess && (e = run_pass(c, 1, o2, 1)) == cudaSuccess &&
        (e = run_pass(c, 0, o3, 1)) == cudaSuccess && (e = run_pass(c, 1, o4, 1)) == cudaSuccess)
      e = run_pass(c, 2, o5, 1);
    if (e != cudaSuccess) return cuda_check(c, e, "coulomb");
  }
  return SKY_OK;
}

__device__ __forceinline__ void rho0_powers(double r0, double alpha, double& r0a, double& r0am1) {
  if (r0 > 1e-30) {
    r0a = pow(r0, alpha);
    r0am1 = r0a / r0;
  } else {
    r0a = 0.0;
    r0am1 = 0.0;
  }
}

__global__ void k_mean_fields(Couplings cp, const double* tau, const double* divJ,
                              const double* f, int G, double* U, double* B, double* W) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= G) return;
  const double r[2] = {f[p], f[G + p]};
  const double l[2] = {f[2 * G + p], f[3 * G + p]};
  const double t[2] = {tau[p] + tau[G + p], tau[p] - tau[G + p]};
  const double d[2] = {divJ[p] + divJ[G + p], divJ[p] - divJ[G + p]};
  double r0a, r0am1;
  rho0_powers(r[0], cp.alpha, r0a, r0am1);
  const double dd = cp.alpha * r0am1 * (cp.rhoa[0] * r[0] * r[0] + cp.rhoa[1] * r[1] * r[1]);
  double uT[2];
#pragma unroll
  for (int T = 0; T < 2; ++T)
    uT[T] = 2.0 * (cp.rho[T] + cp.rhoa[T] * r0a) * r[T] + cp.tau[T] * t[T] +
            2.0 * cp.drho[T] * l[T] + cp.nJ[T] * d[T];
  const double vc = cp.coulomb ? f[10 * G + p] : 0.0;
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const double s1 = q == 0 ? 1.0 : -1.0;
    U[q * G + p] = uT[0] + s1 * uT[1] + dd + (q == 1 ? vc : 0.0);
    B[q * G + p] = cp.hb2m[q] + cp.tau[0] * r[0] + s1 * cp.tau[1] * r[1];
#pragma unroll
    for (int j = 0; j < 3; ++j)
      W[(q * 3 + j) * G + p] = -(cp.nJ[0] * f[(4 + 2 * j) * G + p] +
                                 s1 * cp.nJ[1] * f[(5 + 2 * j) * G + p]);
  }
}

sky_status mean_fields_impl(Ctx* c, const double* rho, const double* tau, const double* divJ,
                            double* U, double* B, double* W) {
  sky_status s = field_prep(c, rho, true);
  if (s != SKY_OK) return s;
  k_mean_fields<<<div_up(c->G, 256), 256, 0, c->stream>>>(c->cp, tau, divJ, c->d_ftmp, c->G, U,
                                                          B, W); note_launch();
  return cuda_check(c, cudaGetLastError(), "mean fields");
}

// ------------------------------------------------------------ energy
constexpr int kEnBlock = 256;
constexpr int kEnParts = 7;   // kin, rho, tau, drho, nJ, coul, A

__global__ void __launch_bounds__(kEnBlock) k_energy_parts(Couplings cp, const double* rho,
                                                           const double* tau,
                                                           const double* divJ,
                                                           const double* f, int G,
                                                           double* part) {
  double acc[kEnParts] = {0, 0, 0, 0, 0, 0, 0};
  for (int p = blockIdx.x * kEnBlock + threadIdx.x; p < G; p += gridDim.x * kEnBlock) {
    const double r[2] = {f[p], f[G + p]};
    const double l[2] = {f[2 * G + p], f[3 * G + p]};
    const double t[2] = {tau[p] + tau[G + p], tau[p] - tau[G + p]};
    const double d[2] = {divJ[p] + divJ[G + p], divJ[p] - divJ[G + p]};
    double r0a, r0am1;
    rho0_powers(r[0], cp.alpha, r0a, r0am1);
    acc[0] += cp.hb2m[0] * tau[p] + cp.hb2m[1] * tau[G + p];
#pragma unroll
    for (int T = 0; T < 2; ++T) {
      acc[1] += (cp.rho[T] + cp.rhoa[T] * r0a) * r[T] * r[T];
      acc[2] += cp.tau[T] * r[T] * t[T];
      acc[3] += cp.drho[T] * r[T] * l[T];
      acc[4] += cp.nJ[T] * r[T] * d[T];
    }
    if (cp.coulomb) acc[5] += 0.5 * rho[G + p] * f[10 * G + p];
    acc[6] += rho[p] + rho[G + p];
  }
  __shared__ double sh[kEnBlock / 32][kEnParts];
#pragma unroll
  for (int k = 0; k < kEnParts; ++k) {
    double v = acc[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5][k] = v;
  }
  __syncthreads();
  if (threadIdx.x < kEnParts) {
    double v = 0.0;
    for (int w = 0; w < kEnBlock / 32; ++w) v += sh[w][threadIdx.x];
    part[blockIdx.x * kEnParts + threadIdx.x] = v;
  }
}

__global__ void k_energy_final(const double* part, int nblk, double dV, double* out, int* status) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double s[kEnParts] = {0, 0, 0, 0, 0, 0, 0};
  for (int b = 0; b < nblk; ++b)
    for (int k = 0; k < kEnParts; ++k) s[k] += part[b * kEnParts + k];
  double tot = 0.0;
  for (int k = 0; k < 6; ++k) {
    out[1 + k] = dV * s[k];
    tot += dV * s[k];
  }
  out[0] = tot;
  out[7] = dV * s[6];
  if (!isfinite(tot)) flag_status(status, SKY_ENAN);
}

sky_status energy_impl(Ctx* c, const double* rho, const double* tau, const double* divJ,
                       double* out) {
  sky_status s = field_prep(c, rho, false);
  if (s != SKY_OK) return s;
  const int nblk = 64;
  double* part = c->d_ftmp + 11 * (long long)c->G;
  k_energy_parts<<<nblk, kEnBlock, 0, c->stream>>>(c->cp, rho, tau, divJ, c->d_ftmp, c->G, part); note_launch();
  k_energy_final<<<1, 32, 0, c->stream>>>(part, nblk, c->dV, out, c->d_status); note_launch();
  return cuda_check(c, cudaGetLastError(), "energy");
}

// ------------------------------------------------------------ convergence
__global__ void k_sp_spread(const double* eps, const double* hn2, int A, double* out) {
  __shared__ double sa[32], sb[32];
  double a = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < A; i += blockDim.x) {
    a += hn2[i] - eps[i] * eps[i];
    b += eps[i];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
  }
  if ((threadIdx.x & 31) == 0) { sa[threadIdx.x >> 5] = a; sb[threadIdx.x >> 5] = b; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double x = 0.0, y = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { x += sa[w]; y += sb[w]; }
    out[0] = A > 0 ? sqrt(fmax(x, 0.0) / A) : 0.0;
    out[1] = y;
  }
}

sky_status sp_spread_impl(Ctx* c, const double* eps, const double* hn2, int A, double* out) {
  k_sp_spread<<<1, 1024, 0, c->stream>>>(eps, hn2, A, out); note_launch();
  return cuda_check(c, cudaGetLastError(), "sp spread");
}

}  // namespace sky
