// FP64 Hermitian eigensolver for steps 3b-3c (Sec. 3.3.2) and the Loewdin /
// Rayleigh-Ritz factors built on it.
//
// The paper diagonalises with ScaLAPACK's tridiagonal + MRRR solver.  Here
// the solver is a parallel cyclic Jacobi method: in each round the indices
// are paired by a round-robin tournament, every pair (p, q) gets the 2x2
// unitary J = D R (D removes the phase of A_pq, R is the real Jacobi
// rotation), and all (I/2)^2 2x2 blocks are updated at once as
// A'[P1,P2] = J1^H A[P1,P2] J2 (ping-pong buffers), with the rotations
// accumulated into V.  One sweep is I-1 rounds; sweeps stop when the
// off-diagonal Frobenius norm falls below tol * ||A||_F.  The whole solve is
// one cooperative kernel whose rounds are separated by a grid barrier with a
// bounded wait.  Near convergence the matrices are close to diagonal and a
// sweep or two suffices.
#include "sky_internal.cuh"

namespace sky {

constexpr int kJacThreads = 256;
constexpr int kJacTile = 16;                  // 16 x 16 work items per tile
constexpr long long kBarrierSpins = 20000000; // x ~64 ns: bounded wait per barrier

struct Rot {
  double c, s;    // real rotation
  double2 e;      // phase of A_pq (unit modulus)
};

// Round-robin pairing: L_r[0] = 0, L_r[i] = 1 + ((i - 1 + r) mod (m - 1)).
__device__ __forceinline__ void pair_of(int k, int r, int m, int& p, int& q) {
  const int i = k, j = m - 1 - k;
  p = (i == 0) ? 0 : 1 + ((i - 1 + r) % (m - 1));
  q = 1 + ((j - 1 + r) % (m - 1));
  if (p > q) { const int t = p; p = q; q = t; }
}

__device__ __forceinline__ Rot make_rot(const double2* A, int m, int n, int p, int q) {
  Rot R;
  R.c = 1.0; R.s = 0.0; R.e = make_double2(1.0, 0.0);
  if (p >= n || q >= n) return R;   // padding index: identity
  const double2 z = A[(long long)p * m + q];
  const double az = hypot(z.x, z.y);
  if (az == 0.0) return R;
  const double app = A[(long long)p * m + p].x, aqq = A[(long long)q * m + q].x;
  const double th = (aqq - app) / (2.0 * az);
  double t;
  if (fabs(th) > 1e150) t = 0.5 / th;
  else t = (th >= 0.0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
  R.c = 1.0 / sqrt(t * t + 1.0);
  R.s = t * R.c;
  R.e = make_double2(z.x / az, z.y / az);
  return R;
}

// J = [[c, s], [-s conj(e), c conj(e)]];  J^H = [[c, -s e], [s, c e]].
__device__ __forceinline__ void block_update(const Rot& R1, const Rot& R2, double2 b00,
                                             double2 b01, double2 b10, double2 b11,
                                             double2& o00, double2& o01, double2& o10,
                                             double2& o11) {
  const double2 ce2 = conjx(R2.e);
  // T = B J2
  const double2 t00 = R2.c * b00 - R2.s * cmul(b01, ce2);
  const double2 t01 = R2.s * b00 + R2.c * cmul(b01, ce2);
  const double2 t10 = R2.c * b10 - R2.s * cmul(b11, ce2);
  const double2 t11 = R2.s * b10 + R2.c * cmul(b11, ce2);
  // B' = J1^H T
  o00 = R1.c * t00 - R1.s * cmul(R1.e, t10);
  o01 = R1.c * t01 - R1.s * cmul(R1.e, t11);
  o10 = R1.s * t00 + R1.c * cmul(R1.e, t10);
  o11 = R1.s * t01 + R1.c * cmul(R1.e, t11);
}

// Sense-free generation barrier over all blocks of a cooperative launch,
// with a bounded spin.  Returns false (and flags SKY_ETIMEOUT) on timeout.
__device__ __forceinline__ bool grid_barrier(unsigned* bar, int* status) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* gen = bar + 1;
    const unsigned my_gen = *gen;
    __threadfence();
    const unsigned arrived = atomicAdd(bar, 1u);
    int ok = 1;
    if (arrived == gridDim.x - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      long long spins = 0;
      while (*gen == my_gen) {
        if (++spins > kBarrierSpins || (*(volatile int*)status & SKY_STATUS_BIT(SKY_ETIMEOUT))) {
          flag_status(status, SKY_ETIMEOUT);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

struct JacArgs {
  double2* A0; double2* A1; double2* V;
  int n, m;
  double tol;
  int max_sweeps;
  double* part;       // [gridDim.x][2]
  unsigned* bar;
  int* status;
  int* result;        // 0: A0 holds the result, 1: A1
};

__global__ void __launch_bounds__(kJacThreads) k_jacobi(JacArgs a) {
  const int m = a.m, n = a.n, h = m / 2;
  double2* cur = a.A0;
  double2* nxt = a.A1;
  int which = 0;
  __shared__ Rot s_r1[kJacTile], s_r2[kJacTile];
  __shared__ double s_red[2][kJacThreads / 32];
  const int ntA = (h + kJacTile - 1) / kJacTile;          // pair tiles per side
  const int ntV = (m + kJacTile - 1) / kJacTile;          // row tiles of V
  const int tilesA = ntA * ntA, tilesV = ntV * ntA;
  for (int sweep = 0;; ++sweep) {
    // off-diagonal and total Frobenius norms of cur
    double off = 0.0, tot = 0.0;
    for (long long e = (long long)blockIdx.x * kJacThreads + threadIdx.x; e < (long long)n * n;
         e += (long long)gridDim.x * kJacThreads) {
      const int i = (int)(e / n), j = (int)(e % n);
      const double2 v = cur[(long long)i * m + j];
      const double w = v.x * v.x + v.y * v.y;
      tot += w;
      if (i != j) off += w;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      off += __shfl_down_sync(0xffffffffu, off, o);
      tot += __shfl_down_sync(0xffffffffu, tot, o);
    }
    if ((threadIdx.x & 31) == 0) {
      s_red[0][threadIdx.x >> 5] = off;
      s_red[1][threadIdx.x >> 5] = tot;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double x = 0.0, y = 0.0;
      for (int w = 0; w < kJacThreads / 32; ++w) { x += s_red[0][w]; y += s_red[1][w]; }
      a.part[2 * blockIdx.x] = x;
      a.part[2 * blockIdx.x + 1] = y;
    }
    if (!grid_barrier(a.bar, a.status)) return;
    __shared__ int s_stop;
    if (threadIdx.x == 0) {
      double x = 0.0, y = 0.0;
      for (int b = 0; b < (int)gridDim.x; ++b) { x += a.part[2 * b]; y += a.part[2 * b + 1]; }
      int stop = (x <= a.tol * a.tol * y) || (y == 0.0);
      if (!stop && sweep >= a.max_sweeps) {
        flag_status(a.status, SKY_ENOCONV);
        stop = 1;
      }
      s_stop = stop;
    }
    __syncthreads();
    if (s_stop) break;
    // the partial norms are rewritten next sweep only after everyone read them
    if (!grid_barrier(a.bar, a.status)) return;
    for (int r = 0; r < m - 1; ++r) {
      for (int t = blockIdx.x; t < tilesA + tilesV; t += gridDim.x) {
        int k1b, k2b, rowb = 0;
        const bool isA = t < tilesA;
        if (isA) { k1b = (t / ntA) * kJacTile; k2b = (t % ntA) * kJacTile; }
        else { const int u = t - tilesA; rowb = (u / ntA) * kJacTile; k2b = (u % ntA) * kJacTile; k1b = 0; }
        __syncthreads();
        if (threadIdx.x < kJacTile) {
          const int k = k2b + threadIdx.x;
          if (k < h) { int p, q; pair_of(k, r, m, p, q); s_r2[threadIdx.x] = make_rot(cur, m, n, p, q); }
        } else if (isA && threadIdx.x < 2 * kJacTile) {
          const int k = k1b + threadIdx.x - kJacTile;
          if (k < h) { int p, q; pair_of(k, r, m, p, q); s_r1[threadIdx.x - kJacTile] = make_rot(cur, m, n, p, q); }
        }
        __syncthreads();
        const int ia = threadIdx.x / kJacTile, ib = threadIdx.x % kJacTile;
        if (isA) {
          const int k1 = k1b + ia, k2 = k2b + ib;
          if (k1 < h && k2 < h) {
            int p1, q1, p2, q2;
            pair_of(k1, r, m, p1, q1);
            pair_of(k2, r, m, p2, q2);
            const Rot& R1 = s_r1[ia];
            const Rot& R2 = s_r2[ib];
            double2 o00, o01, o10, o11;
            if (k1 == k2 && p1 < n && q1 < n && (R1.s != 0.0 || R1.e.y != 0.0 || R1.e.x != 1.0)) {
              // diagonal block: exact result of the 2x2 diagonalisation
              const double2 z = cur[(long long)p1 * m + q1];
              const double az = hypot(z.x, z.y);
              const double t = R1.s / R1.c;
              o00 = make_double2(cur[(long long)p1 * m + p1].x - t * az, 0.0);
              o11 = make_double2(cur[(long long)q1 * m + q1].x + t * az, 0.0);
              o01 = make_double2(0.0, 0.0);
              o10 = o01;
            } else {
              block_update(R1, R2, cur[(long long)p1 * m + p2], cur[(long long)p1 * m + q2],
                           cur[(long long)q1 * m + p2], cur[(long long)q1 * m + q2], o00, o01, o10,
                           o11);
            }
            nxt[(long long)p1 * m + p2] = o00;
            nxt[(long long)p1 * m + q2] = o01;
            nxt[(long long)q1 * m + p2] = o10;
            nxt[(long long)q1 * m + q2] = o11;
          }
        } else {
          const int row = rowb + ia, k = k2b + ib;
          if (row < m && k < h) {
            int p, q;
            pair_of(k, r, m, p, q);
            const Rot& R = s_r2[ib];
            const double2 vp = a.V[(long long)row * m + p], vq = a.V[(long long)row * m + q];
            const double2 ce = conjx(R.e);
            a.V[(long long)row * m + p] = R.c * vp - R.s * cmul(vq, ce);
            a.V[(long long)row * m + q] = R.s * vp + R.c * cmul(vq, ce);
          }
        }
      }
      if (!grid_barrier(a.bar, a.status)) return;
      double2* tmp = cur; cur = nxt; nxt = tmp;
      which ^= 1;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *a.result = which;
}

// Copy A (n x n) into the padded m x m buffer, V = identity, reset the barrier.
__global__ void k_jacobi_init(const double2* A, int n, int m, double2* A0, double2* V,
                              unsigned* bar, int* result) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e == 0) { bar[0] = 0u; *result = 0; }
  if (e >= (long long)m * m) return;
  const int i = (int)(e / m), j = (int)(e % m);
  A0[e] = (i < n && j < n) ? A[(long long)i * n + j] : make_double2(0.0, 0.0);
  V[e] = make_double2(i == j ? 1.0 : 0.0, 0.0);
}

// Eigenvalues ascending (ties by index) and the matching columns of V.
__global__ void k_jacobi_finish(const double2* A0, const double2* A1, const double2* V,
                                const int* result, int n, int m, double* w, double2* Z) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const double2* A = (*result) ? A1 : A0;
  const double dj = A[(long long)j * m + j].x;
  int rank = 0;
  for (int i = 0; i < n; ++i) {
    const double di = A[(long long)i * m + i].x;
    rank += (di < dj) || (di == dj && i < j);
  }
  w[rank] = dj;
  for (int i = 0; i < n; ++i) Z[(long long)i * n + rank] = V[(long long)i * m + j];
}

int jacobi_max_grid(Ctx* c) {
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_jacobi, kJacThreads, 0);
  if (per_sm < 1) per_sm = 1;
  return per_sm * c->num_sms;
}

sky_status eigh_impl(Ctx* c, const double2* A, int I, double* w, double2* Z) {
  if (I == 0) return SKY_OK;
  const int m = I + (I & 1);
  k_jacobi_init<<<div_up((long long)m * m, 256), 256, 0, c->stream>>>(A, I, m, c->d_eigA[0],
                                                                      c->d_eigV, c->d_bar,
                                                                      c->d_eigres); note_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_check(c, e, "jacobi init");
  if (m >= 2) {
    const int h = m / 2;
    const int ntA = (h + kJacTile - 1) / kJacTile, ntV = (m + kJacTile - 1) / kJacTile;
    int grid = ntA * ntA + ntV * ntA;
    if (grid > c->eig_grid) grid = c->eig_grid;
    JacArgs a;
    a.A0 = c->d_eigA[0]; a.A1 = c->d_eigA[1]; a.V = c->d_eigV;
    a.n = I; a.m = m;
    a.tol = 1e-15;
    a.max_sweeps = 60;
    a.part = c->d_eigpart; a.bar = c->d_bar; a.status = c->d_status; a.result = c->d_eigres;
    void* args[] = {&a};
    note_launch();
    e = cudaLaunchCooperativeKernel((const void*)k_jacobi, dim3(grid), dim3(kJacThreads), args, 0,
                                    c->stream);
    if (e != cudaSuccess) return cuda_check(c, e, "jacobi");
  }
  k_jacobi_finish<<<div_up(I, 128), 128, 0, c->stream>>>(c->d_eigA[0], c->d_eigA[1], c->d_eigV,
                                                        c->d_eigres, I, m, w, Z); note_launch();
  return cuda_check(c, cudaGetLastError(), "jacobi finish");
}

// Y = X diag(lambda^{-1/2}); flags SKY_ENOTPD for a non-positive eigenvalue.
__global__ void k_inv_sqrt_cols(const double2* X, const double* lam, int n, double2* Y, int* status) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)n * n) return;
  const int j = (int)(e % n);
  double l = lam[j];
  if (!(l > 0.0)) {
    if (e == j) flag_status(status, SKY_ENOTPD);
    l = 1e-300;
  }
  Y[e] = (1.0 / sqrt(l)) * X[e];
}

// H' = (H' + H'^H) / 2 in place.
__global__ void k_hermitize(double2* A, int n) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)n * n) return;
  const int i = (int)(e / n), j = (int)(e % n);
  if (i > j) return;
  const double2 a = A[(long long)i * n + j], b = A[(long long)j * n + i];
  const double2 s = 0.5 * (a + conjx(b));
  A[(long long)i * n + j] = s;
  A[(long long)j * n + i] = conjx(s);
}

sky_status lowdin_impl(Ctx* c, const double2* S, int I, double2* C) {
  if (I == 0) return SKY_OK;
  double2* X = c->d_small[0];
  double2* Y = c->d_small[1];
  sky_status st = eigh_impl(c, S, I, c->d_eigw, X);
  if (st != SKY_OK) return st;
  k_inv_sqrt_cols<<<div_up((long long)I * I, 256), 256, 0, c->stream>>>(X, c->d_eigw, I, Y,
                                                                       c->d_status); note_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_check(c, e, "loewdin scale");
  return zgemm_small(c, false, true, Y, X, C, I);   // C = Y X^H
}

sky_status subspace_impl(Ctx* c, const double2* H, const double2* C, int I, double2* M,
                         double* eps) {
  if (I == 0) return SKY_OK;
  double2* T1 = c->d_small[0];
  double2* Hp = c->d_small[1];
  double2* Z = c->d_small[2];
  sky_status st = zgemm_small(c, true, false, C, H, T1, I);   // C^H H
  if (st == SKY_OK) st = zgemm_small(c, false, false, T1, C, Hp, I);   // (C^H H) C
  if (st != SKY_OK) return st;
  k_hermitize<<<div_up((long long)I * I, 256), 256, 0, c->stream>>>(Hp, I); note_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_check(c, e, "hermitize");
  st = eigh_impl(c, Hp, I, eps, Z);
  if (st != SKY_OK) return st;
  return zgemm_small(c, false, false, C, Z, M, I);   // M = C Z
}

}  // namespace sky
