// Learned damping weight of the damped gradient step (an extension of
// Sec. 2.2, Eq. dampstep): a periodic 3x3x3 convolutional network
//   x = (U/50, B/hb2m - 1, |W|/5) -> tanh conv 16 -> tanh conv 16 -> conv 1
//   w = WMAX sigmoid(z)
// with its training kernels: the per-voxel statistics of the one-step loss,
// the backward pass through the three layers, and Adam.
//
// Layout: every activation is channel-planar [C][nz][ny][nx] float, x
// fastest, so neighbouring threads read neighbouring voxels.  One thread
// computes all output channels of one voxel; the layer's weights sit in
// shared memory and are read as broadcasts.  Weight gradients are summed per
// (output, input) channel pair over a voxel range by one block, then over the
// ranges in a fixed order, so every result is deterministic.
#include "sky_internal.cuh"

namespace sky {

constexpr int kH = SKY_NET_HIDDEN;
constexpr int kConvThreads = 128;
constexpr int kWgThreads = 256;
constexpr int kMaxSplits = 16;
constexpr int kTaps = 27;
// parameter offsets (the order of the flat vector)
constexpr int oW1 = 0, ob1 = oW1 + kH * 3 * kTaps, oW2 = ob1 + kH, ob2 = oW2 + kH * kH * kTaps,
              oW3 = ob2 + kH, ob3 = oW3 + kH * kTaps, kNParam = ob3 + 1;
static_assert(kNParam == SKY_NET_NPARAM, "parameter count");
// workspace offsets in units of G floats
constexpr int wsX = 0, wsH1 = 3, wsH2 = wsH1 + kH, wsW = wsH2 + kH, wsDZ = wsW + 1,
              wsD2 = wsDZ + 1, wsD1 = wsD2 + kH, wsEnd = wsD1 + kH;
static_assert(wsEnd <= SKY_NET_WS_PER_POINT, "workspace per grid point");

size_t net_partial_elems(int G) {
  const size_t wg = (size_t)kH * kH * kMaxSplits * 28;
  const size_t red = (size_t)div_up(G, kConvThreads) + 8;
  return wg > red ? wg : red;
}

// Periodic neighbour offsets of voxel p: xs[k], ys[k], zs[k] for d = k - 1,
// ys and zs already multiplied by their strides.
struct Nbr {
  int xs[3], ys[3], zs[3];
  __device__ __forceinline__ int z(int a) const { return a == 0 ? zs[0] : (a == 1 ? zs[1] : zs[2]); }
  __device__ __forceinline__ Nbr(int p, int nx, int ny, int nz) {
    const int x = p % nx, y = (p / nx) % ny, z = p / (nx * ny);
    xs[0] = x == 0 ? nx - 1 : x - 1; xs[1] = x; xs[2] = x == nx - 1 ? 0 : x + 1;
    ys[0] = (y == 0 ? ny - 1 : y - 1) * nx; ys[1] = y * nx; ys[2] = (y == ny - 1 ? 0 : y + 1) * nx;
    const int s = nx * ny;
    zs[0] = (z == 0 ? nz - 1 : z - 1) * s; zs[1] = z * s; zs[2] = (z == nz - 1 ? 0 : z + 1) * s;
  }
};

__global__ void k_net_features(const double* __restrict__ U, const double* __restrict__ B,
                               const double* __restrict__ W, int G, double hb2m, float* __restrict__ x) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= G) return;
  const double wx = W[p], wy = W[G + p], wz = W[2 * G + p];
  x[p] = (float)(U[p] / SKY_NET_USCALE);
  x[G + p] = (float)(B[p] / hb2m - 1.0);
  x[2 * G + p] = (float)(sqrt(wx * wx + wy * wy + wz * wz) / SKY_NET_WSCALE);
}

// out_o(r) = b_o + sum_{i,d} W[o][i][t(d)] in_i(r + d); ACT 0: tanh, 1: the
// weight: out = WMAX sigmoid (the network's own output) and
// wout = 1 + scale (out - 1) (the weight the step uses).
template <int CIN, int COUT, int ACT>
__global__ void __launch_bounds__(kConvThreads) k_conv_fwd(const float* __restrict__ in,
                                                           const float* __restrict__ Wt,
                                                           const float* __restrict__ bias,
                                                           float* __restrict__ out, int nx, int ny,
                                                           int nz, float* __restrict__ wout = nullptr,
                                                           float scale = 1.0f) {
  __shared__ float sw[COUT * CIN * kTaps];
  for (int i = threadIdx.x; i < COUT * CIN * kTaps; i += blockDim.x) sw[i] = Wt[i];
  __syncthreads();
  const int G = nx * ny * nz;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= G) return;
  const Nbr nb(p, nx, ny, nz);
  float acc[COUT];
#pragma unroll
  for (int o = 0; o < COUT; ++o) acc[o] = bias[o];
#pragma unroll 1
  for (int a = 0; a < 3; ++a) {
    const int za = nb.z(a);
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const int t = 9 * a + 3 * b + c;
        const int q = za + nb.ys[b] + nb.xs[c];
#pragma unroll (CIN < 4 ? CIN : 4)
        for (int i = 0; i < CIN; ++i) {
          const float v = __ldg(in + (size_t)i * G + q);
#pragma unroll
          for (int o = 0; o < COUT; ++o) acc[o] = fmaf(sw[(o * CIN + i) * kTaps + t], v, acc[o]);
        }
      }
  }
#pragma unroll
  for (int o = 0; o < COUT; ++o) {
    if (ACT == 0) {
      out[(size_t)o * G + p] = tanhf(acc[o]);
    } else {
      const float w = (float)SKY_NET_WMAX / (1.0f + expf(-acc[o]));
      out[(size_t)o * G + p] = w;
      wout[p] = 1.0f + scale * (w - 1.0f);
    }
  }
}

// din_i(r) = (1 - hin_i(r)^2) sum_{o,d} W[o][i][t(d)] dout_o(r - d).
template <int CIN, int COUT>
__global__ void __launch_bounds__(kConvThreads) k_conv_bwd_in(const float* __restrict__ dout,
                                                              const float* __restrict__ Wt,
                                                              const float* __restrict__ hin,
                                                              float* __restrict__ din, int nx,
                                                              int ny, int nz) {
  __shared__ float sw[COUT * CIN * kTaps];
  for (int i = threadIdx.x; i < COUT * CIN * kTaps; i += blockDim.x) sw[i] = Wt[i];
  __syncthreads();
  const int G = nx * ny * nz;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= G) return;
  const Nbr nb(p, nx, ny, nz);
  float acc[CIN];
#pragma unroll
  for (int i = 0; i < CIN; ++i) acc[i] = 0.0f;
#pragma unroll 1
  for (int a = 0; a < 3; ++a) {
    const int za = nb.z(2 - a);
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const int t = 9 * a + 3 * b + c;
        const int q = za + nb.ys[2 - b] + nb.xs[2 - c];   // r - d
#pragma unroll (COUT < 4 ? COUT : 4)
        for (int o = 0; o < COUT; ++o) {
          const float v = __ldg(dout + (size_t)o * G + q);
#pragma unroll
          for (int i = 0; i < CIN; ++i) acc[i] = fmaf(sw[(o * CIN + i) * kTaps + t], v, acc[i]);
        }
      }
  }
#pragma unroll
  for (int i = 0; i < CIN; ++i) {
    const float h = hin[(size_t)i * G + p];
    din[(size_t)i * G + p] = acc[i] * (1.0f - h * h);
  }
}

// part[(pair * nsplit + split) * 28 + t] = sum over the split's voxels of
// dout_o(r) in_i(r + d_t) (t < 27) and dout_o(r) (t = 27); pair = o * CIN + i.
template <int CIN>
__global__ void __launch_bounds__(kWgThreads) k_conv_wgrad(const float* __restrict__ dout,
                                                           const float* __restrict__ in, int nx,
                                                           int ny, int nz, int chunk,
                                                           double* __restrict__ part) {
  const int pair = blockIdx.x, o = pair / CIN, i = pair % CIN;
  const int G = nx * ny * nz;
  const int p0 = blockIdx.y * chunk, p1 = min(G, p0 + chunk);
  float acc[28];
#pragma unroll
  for (int t = 0; t < 28; ++t) acc[t] = 0.0f;
  const float* di = dout + (size_t)o * G;
  const float* xi = in + (size_t)i * G;
  for (int p = p0 + threadIdx.x; p < p1; p += blockDim.x) {
    const float v = di[p];
    const Nbr nb(p, nx, ny, nz);
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b)
#pragma unroll
        for (int c = 0; c < 3; ++c)
          acc[9 * a + 3 * b + c] = fmaf(v, __ldg(xi + nb.zs[a] + nb.ys[b] + nb.xs[c]), acc[9 * a + 3 * b + c]);
    acc[27] += v;
  }
  __shared__ double sred[kWgThreads / 32][28];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int t = 0; t < 28; ++t) {
    float s = acc[t];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (lane == 0) sred[warp][t] = (double)s;
  }
  __syncthreads();
  if (threadIdx.x < 28) {
    double s = 0.0;
    for (int w = 0; w < kWgThreads / 32; ++w) s += sred[w][threadIdx.x];
    part[((size_t)pair * gridDim.y + blockIdx.y) * 28 + threadIdx.x] = s;
  }
}

// grad[oW + pair * 27 + t] += sum_split part; grad[ob + o] += bias part of pair (o, 0).
__global__ void k_wgrad_reduce(const double* __restrict__ part, int nsplit, int cin,
                               double* __restrict__ gW, double* __restrict__ gb) {
  const int pair = blockIdx.x, t = threadIdx.x;
  if (t >= 28) return;
  double s = 0.0;
  for (int k = 0; k < nsplit; ++k) s += part[((size_t)pair * nsplit + k) * 28 + t];
  if (t < kTaps) gW[(size_t)pair * kTaps + t] += s;
  else if (pair % cin == 0) gb[pair / cin] += s;
}

template <int NT>
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double red[NT / 32];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int k = 0; k < NT / 32; ++k) s += red[k];
  return s;
}

// dz(r) = d L / d z(r) with L = sum (a w^2 - 2 b w + c) / norm and
// w = WMAX sigmoid(z); block partials of the unnormalised loss.
__global__ void __launch_bounds__(kConvThreads) k_net_head(const float* __restrict__ w,
                                                           const double* __restrict__ abc,
                                                           const double* __restrict__ norm, int G,
                                                           float* __restrict__ dz,
                                                           double* __restrict__ lpart) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  double l = 0.0;
  if (p < G) {
    const double a = abc[p], b = abc[G + p], c = abc[2 * G + p], ww = w[p];
    const double dw = 2.0 * (a * ww - b) / norm[0];
    dz[p] = (float)(dw * ww * (1.0 - ww / SKY_NET_WMAX));
    l = a * ww * ww - 2.0 * b * ww + c;
  }
  l = block_sum<kConvThreads>(l);
  if (threadIdx.x == 0) lpart[blockIdx.x] = l;
}

__global__ void k_loss_total(const double* __restrict__ lpart, int nblk,
                             const double* __restrict__ norm, double* __restrict__ loss) {
  double s = 0.0;
  for (int k = threadIdx.x; k < nblk; k += blockDim.x) s += lpart[k];
  s = block_sum<256>(s);
  if (threadIdx.x == 0) loss[0] += s / norm[0];
}

__global__ void k_adam(float* __restrict__ theta, double* __restrict__ grad,
                       double* __restrict__ m, double* __restrict__ v, int n, double lr,
                       double b1, double b2, double eps, double c1, double c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double g = grad[i];
  const double mi = b1 * m[i] + (1.0 - b1) * g;
  const double vi = b2 * v[i] + (1.0 - b2) * g * g;
  m[i] = mi;
  v[i] = vi;
  theta[i] = (float)((double)theta[i] - lr * (mi / c1) / (sqrt(vi / c2) + eps));
  grad[i] = 0.0;
}

// a = sum |psi - phi|^2, b = sum Re(conj(psi - phi)(psi - ppsi)),
// c = sum |psi - ppsi|^2 over states and spin, per voxel; block partials of c.
template <typename T>
__global__ void __launch_bounds__(kConvThreads) k_precond_stats(const cx<T>* __restrict__ psi,
                                                                const cx<T>* __restrict__ phi,
                                                                const cx<T>* __restrict__ pp,
                                                                int I, int G,
                                                                double* __restrict__ abc,
                                                                double* __restrict__ cpart) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  double a = 0.0, b = 0.0, c = 0.0;
  if (p < G) {
    for (long long k = 0; k < 2LL * I; ++k) {
      const long long o = k * G + p;
      const double2 s = to_d2(psi[o]), f = to_d2(phi[o]), r = to_d2(pp[o]);
      const double gx = s.x - f.x, gy = s.y - f.y, dx = s.x - r.x, dy = s.y - r.y;
      a += gx * gx + gy * gy;
      b += gx * dx + gy * dy;
      c += dx * dx + dy * dy;
    }
    abc[p] = a;
    abc[G + p] = b;
    abc[2 * G + p] = c;
  }
  c = block_sum<kConvThreads>(c);
  if (threadIdx.x == 0) cpart[blockIdx.x] = c;
}

__global__ void k_norm_total(const double* __restrict__ cpart, int nblk, double* __restrict__ norm) {
  double s = 0.0;
  for (int k = threadIdx.x; k < nblk; k += blockDim.x) s += cpart[k];
  s = block_sum<256>(s);
  if (threadIdx.x == 0) norm[0] = s;
}

// ------------------------------------------------------------ host side
sky_status net_forward_impl(Ctx* c, int q, const float* theta, const double* U, const double* B,
                            const double* W, double scale, float* ws, float* w) {
  const int G = c->G, nx = c->n[0], ny = c->n[1], nz = c->n[2];
  const unsigned nb = div_up(G, kConvThreads);
  float* x = ws + (size_t)wsX * G;
  float* h1 = ws + (size_t)wsH1 * G;
  float* h2 = ws + (size_t)wsH2 * G;
  k_net_features<<<nb, kConvThreads, 0, c->stream>>>(U, B, W, G, c->cp.hb2m[q], x);
  k_conv_fwd<3, kH, 0><<<nb, kConvThreads, 0, c->stream>>>(x, theta + oW1, theta + ob1, h1, nx, ny, nz);
  k_conv_fwd<kH, kH, 0><<<nb, kConvThreads, 0, c->stream>>>(h1, theta + oW2, theta + ob2, h2, nx, ny, nz);
  k_conv_fwd<kH, 1, 1><<<nb, kConvThreads, 0, c->stream>>>(h2, theta + oW3, theta + ob3,
                                                            ws + (size_t)wsW * G, nx, ny, nz, w,
                                                            (float)scale);
  note_launch(4);
  return cuda_check(c, cudaGetLastError(), "net forward");
}

template <int CIN>
static cudaError_t wgrad(Ctx* c, int cout, const float* dout, const float* in, double* gW,
                         double* gb) {
  const int G = c->G;
  const int pairs = cout * CIN;
  int ns = (2 * c->num_sms + pairs - 1) / pairs;
  if (ns > kMaxSplits) ns = kMaxSplits;
  const int maxns = (int)div_up(G, kWgThreads);
  if (ns > maxns) ns = maxns;
  if (ns < 1) ns = 1;
  const int chunk = (int)div_up(G, ns);
  k_conv_wgrad<CIN><<<dim3(pairs, ns), kWgThreads, 0, c->stream>>>(dout, in, c->n[0], c->n[1],
                                                                   c->n[2], chunk, c->d_netpart);
  k_wgrad_reduce<<<pairs, 32, 0, c->stream>>>(c->d_netpart, ns, CIN, gW, gb);
  note_launch(2);
  return cudaGetLastError();
}

sky_status net_backward_impl(Ctx* c, const float* theta, float* ws, const double* abc,
                             const double* norm, double* grad, double* loss) {
  const int G = c->G, nx = c->n[0], ny = c->n[1], nz = c->n[2];
  const unsigned nb = div_up(G, kConvThreads);
  float* x = ws + (size_t)wsX * G;
  float* h1 = ws + (size_t)wsH1 * G;
  float* h2 = ws + (size_t)wsH2 * G;
  const float* w = ws + (size_t)wsW * G;
  float* dz = ws + (size_t)wsDZ * G;
  float* d2 = ws + (size_t)wsD2 * G;
  float* d1 = ws + (size_t)wsD1 * G;
  k_net_head<<<nb, kConvThreads, 0, c->stream>>>(w, abc, norm, G, dz, c->d_netpart);
  k_loss_total<<<1, 256, 0, c->stream>>>(c->d_netpart, (int)nb, norm, loss);
  note_launch(2);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = wgrad<kH>(c, 1, dz, h2, grad + oW3, grad + ob3);
  if (e == cudaSuccess) {
    k_conv_bwd_in<kH, 1><<<nb, kConvThreads, 0, c->stream>>>(dz, theta + oW3, h2, d2, nx, ny, nz);
    note_launch();
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = wgrad<kH>(c, kH, d2, h1, grad + oW2, grad + ob2);
  if (e == cudaSuccess) {
    k_conv_bwd_in<kH, kH><<<nb, kConvThreads, 0, c->stream>>>(d2, theta + oW2, h1, d1, nx, ny, nz);
    note_launch();
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = wgrad<3>(c, kH, d1, x, grad + oW1, grad + ob1);
  return cuda_check(c, e, "net backward");
}

sky_status net_adam_impl(Ctx* c, float* theta, double* grad, double* m, double* v, int step,
                         double lr, double beta1, double beta2, double eps) {
  const double c1 = 1.0 - pow(beta1, (double)step), c2 = 1.0 - pow(beta2, (double)step);
  k_adam<<<div_up(kNParam, 256), 256, 0, c->stream>>>(theta, grad, m, v, kNParam, lr, beta1, beta2,
                                                      eps, c1, c2);
  note_launch();
  return cuda_check(c, cudaGetLastError(), "net adam");
}

sky_status precond_stats_impl(Ctx* c, const void* psi, const void* phi, const void* ppsi, int I,
                              double* abc, double* norm) {
  const int G = c->G;
  const unsigned nb = div_up(G, kConvThreads);
  if (c->prec == SKY_F64)
    k_precond_stats<double><<<nb, kConvThreads, 0, c->stream>>>(
        (const double2*)psi, (const double2*)phi, (const double2*)ppsi, I, G, abc, c->d_netpart);
  else
    k_precond_stats<float><<<nb, kConvThreads, 0, c->stream>>>(
        (const float2*)psi, (const float2*)phi, (const float2*)ppsi, I, G, abc, c->d_netpart);
  k_norm_total<<<1, 256, 0, c->stream>>>(c->d_netpart, (int)nb, norm);
  note_launch(2);
  return cuda_check(c, cudaGetLastError(), "precond stats");
}

}  // namespace sky
