// Time-dependent stepping (Sky3D's time-dependent mode, Sec. 1; Sec. 2.2:
// the time-evolution operator is unitary, so the states stay orthonormal
// with no orthonormalisation, each nucleon evolves on its own and the
// nucleons couple only through the mean field).  The propagator
// exp(-i tau h), tau = dt / hbar, is applied as its Taylor polynomial
//   out = sum_{k=0}^{m} t_k,   t_0 = psi,   t_k = (-i tau / k) h t_{k-1},
// each h t_{k-1} by the h psi kernels of sky_apply_h, each term scaled and
// added to the sum by one fused kernel.  Which mean field the caller passes
// (the predictor-corrector midpoint field, for example) is the caller's.
#include "sky_internal.cuh"

namespace sky {
namespace {

// term <- c term; out <- (first ? psi : out) + term, over n complex values.
template <typename S>
__global__ void __launch_bounds__(256) k_td_term(S* __restrict__ term, S* __restrict__ out,
                                                 const S* __restrict__ psi, long long n, double cr,
                                                 double ci, int first) {
  using R = decltype(S().x);
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const S h = term[e];
  S t;
  t.x = (R)cr * h.x - (R)ci * h.y;
  t.y = (R)cr * h.y + (R)ci * h.x;
  term[e] = t;
  const S base = first ? psi[e] : out[e];
  S o;
  o.x = base.x + t.x;
  o.y = base.y + t.y;
  out[e] = o;
}

template <typename S>
sky_status td_taylor_t(Ctx* c, const double* U, const double* B, const double* W, const S* psi,
                       S* out, S* work, int I, double tau, int order) {
  const long long n = 2LL * c->G * I;
  if (order == 0)
    return cuda_check(c, cudaMemcpyAsync(out, psi, n * sizeof(S), cudaMemcpyDeviceToDevice, c->stream),
                      "td copy");
  const S* src = psi;
  for (int k = 1; k <= order; ++k) {
    S* dst = work + ((k & 1) ? 0 : n);   // ping-pong between the two work halves
    sky_status s = apply_h_impl(c, U, B, W, src, dst, I, nullptr, nullptr);
    if (s != SKY_OK) return s;
    // c_k = -i tau / k
    k_td_term<S><<<div_up(n, 256), 256, 0, c->stream>>>(dst, out, psi, n, 0.0, -tau / k, k == 1);
    note_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_check(c, e, "td term");
    src = dst;
  }
  return SKY_OK;
}

}  // namespace

sky_status td_taylor_impl(Ctx* c, const double* U, const double* B, const double* W,
                          const void* psi, void* out, void* work, int I, double tau, int order) {
  if (c->prec == SKY_F64)
    return td_taylor_t<double2>(c, U, B, W, (const double2*)psi, (double2*)out, (double2*)work, I,
                                tau, order);
  return td_taylor_t<float2>(c, U, B, W, (const float2*)psi, (float2*)out, (float2*)work, I, tau,
                             order);
}

}  // namespace sky
