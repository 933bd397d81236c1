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

constexpr int kJacThreads = 512;
constexpr long long kBarrierSpins = 40000000; // x ~32 ns: bounded wait per barrier

// Rotation of one index pair (p, q) in one round.  J = D R with D removing the
// phase of A_pq and R the real Jacobi rotation:
//   J = [[c, s], [j10, j11]],  j10 = -s ce,  j11 = c ce,  ce = e^{-i arg A_pq};
//   J^H = [[c, conj(j10)], [s, conj(j11)]].
// dp, dq are the new diagonal entries; id marks a rotation skipped because
// |A_pq| is below the threshold (then J = 1).
struct JRot {
  double c, s;
  double2 j10, j11;
  double dp, dq;
  int p, q, id, pad;
};

// a x + b y with a real and b, x, y complex (six FP64 operations).
__device__ __forceinline__ double2 rx_plus_cy(double a, double2 x, double2 b, double2 y) {
  double2 r;
  r.x = fma(b.x, y.x, a * x.x);
  r.x = fma(-b.y, y.y, r.x);
  r.y = fma(b.x, y.y, a * x.y);
  r.y = fma(b.y, y.x, r.y);
  return r;
}
// a x + conj(b) y.
__device__ __forceinline__ double2 rx_plus_conjcy(double a, double2 x, double2 b, double2 y) {
  double2 r;
  r.x = fma(b.x, y.x, a * x.x);
  r.x = fma(b.y, y.y, r.x);
  r.y = fma(b.x, y.y, a * x.y);
  r.y = fma(-b.y, y.x, r.y);
  return r;
}

// Round-robin pairing: L_r[0] = 0, L_r[i] = 1 + ((i - 1 + r) mod (m - 1));
// pair k of round r is (L_r[k], L_r[m-1-k]), returned with p < q.
__device__ __forceinline__ void pair_of(int k, int r, int m, int& p, int& q) {
  const int j = m - 1 - k;
  p = (k == 0) ? 0 : 1 + ((k - 1 + r) % (m - 1));
  q = 1 + ((j - 1 + r) % (m - 1));
  if (p > q) { const int t = p; p = q; q = t; }
}
// Inverse: the pair index of index i in round r.
__device__ __forceinline__ int pair_index(int i, int r, int m) {
  if (i == 0) return 0;
  const int pos = ((i - 1 - r) % (m - 1) + (m - 1)) % (m - 1) + 1;
  return pos < m / 2 ? pos : m - 1 - pos;
}

// x^{-1/2} from an FP32 seed and two Newton steps in FP64, r <- r (3 - x r^2)/2
// (relative error 1e-7 -> 1e-14 -> rounding); x must lie in the FP32 range.
__device__ __forceinline__ double rsqrt_refined(double x) {
  double r = (double)rsqrtf((float)x);
  r = r * fma(-0.5 * x, r * r, 1.5);
  r = r * fma(-0.5 * x, r * r, 1.5);
  return r;
}

// 1/x from an FP32 seed and two Newton steps in FP64, r <- r (2 - x r);
// x must lie in the FP32 range.
__device__ __forceinline__ double rcp_refined(double x) {
  double r = (double)__frcp_rn((float)x);
  r = r * fma(-x, r, 2.0);
  r = r * fma(-x, r, 2.0);
  return r;
}

// Jacobi rotation of B = [[app, z], [z*, aqq]] to FP64 accuracy without the
// FP64 divide, square root and hypot sequences: every reciprocal and
// (inverse) square root starts from an FP32 seed and is refined by Newton
// steps in FP64.  t solves t^2 + 2 theta t - 1 = 0 (smaller root), so the
// rotated pivot is zero to rounding and dp, dq = app -/+ t |z| are the new
// diagonal entries.
__device__ __forceinline__ JRot make_rot(double app, double aqq, double2 z, int p, int q, int n,
                                         double thr) {
  JRot R;
  R.c = 1.0; R.s = 0.0; R.j10 = make_double2(0.0, 0.0); R.j11 = make_double2(1.0, 0.0);
  R.dp = app; R.dq = aqq; R.p = p; R.q = q; R.id = 1; R.pad = 0;
  if (p >= n || q >= n) return R;   // padding index: identity
  const double z2 = z.x * z.x + z.y * z.y;
  if (!(z2 > thr * thr)) return R;
  double rz, az;
  if (z2 > 1e-30 && z2 < 1e30) {
    rz = rsqrt_refined(z2);
    az = z2 * rz;
  } else {
    az = hypot(z.x, z.y);
    rz = 1.0 / az;
  }
  const double th = (aqq - app) * 0.5 * rz;
  const double ath = fabs(th);
  double t;
  if (ath > 1e7) {
    t = 0.5 / th;                               // 1/(2 theta) to rounding here
  } else {
    const double u = fma(th, th, 1.0);
    const double sq = u * rsqrt_refined(u);      // sqrt(theta^2 + 1)
    t = rcp_refined(ath + sq);
    if (th < 0.0) t = -t;
  }
  const double c = rsqrt_refined(fma(t, t, 1.0));
  const double sn = t * c;
  R.c = c;
  R.s = sn;
  const double2 ce = make_double2(z.x * rz, -z.y * rz);
  R.j10 = make_double2(-sn * ce.x, -sn * ce.y);
  R.j11 = make_double2(c * ce.x, c * ce.y);
  R.dp = app - t * az;
  R.dq = aqq + t * az;
  R.id = 0;
  return R;
}

// Column `col` of (B J2) for the 2x2 block B = [[b00, b01], [b10, b11]].
__device__ __forceinline__ void right_col(const JRot& R2, int col, double2 b00, double2 b01,
                                          double2 b10, double2 b11, double2& t0, double2& t1) {
  const double a = col ? R2.s : R2.c;
  const double2 f = col ? R2.j11 : R2.j10;
  t0 = rx_plus_cy(a, b00, f, b01);
  t1 = rx_plus_cy(a, b10, f, b11);
}
// Row `row` of J1^H applied to the column (t0, t1).
__device__ __forceinline__ double2 left_row(const JRot& R1, int row, double2 t0, double2 t1) {
  return row ? rx_plus_conjcy(R1.s, t0, R1.j11, t1) : rx_plus_conjcy(R1.c, t0, R1.j10, t1);
}

// Grid barrier over all blocks of a cooperative launch: a monotonic arrival
// counter (reset before the launch); barrier number e completes when it
// reaches e * gridDim.x.  Release-add to arrive, acquire loads to wait, with
// a bounded spin: on timeout it flags SKY_ETIMEOUT and returns false.
__device__ __forceinline__ bool grid_barrier(unsigned* bar, unsigned& epoch, int* status) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ++epoch;
    const unsigned target = epoch * gridDim.x;
    asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(bar) : "memory");
    int ok = 1;
    long long spins = 0;
    for (;;) {
      unsigned v;
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(bar) : "memory");
      if ((int)(v - target) >= 0) break;
      if (++spins > kBarrierSpins || (*(volatile int*)status & SKY_STATUS_BIT(SKY_ETIMEOUT))) {
        flag_status(status, SKY_ETIMEOUT);
        ok = 0;
        break;
      }
      if (spins > 64) __nanosleep(32);
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

struct JacArgs {
  double2* A0; double2* A1; double2* V;
  JRot* R0; JRot* R1;   // rotations of the current / next round, [m/2] each
  int n, m;
  double tol;
  int max_sweeps;
  double* part;         // [gridDim.x][2]
  unsigned* bar;
  int* status;
  int* result;          // 0: A0 holds the result, 1: A1
  const int* run;       // device gate: skip the whole solve when *run == 0
  long long* stats;     // [0] solves, [1] sweeps in total, [2] sweeps of the last solve
};

__device__ __forceinline__ void block_norms(double off, double tot, double* part) {
  __shared__ double s_red[2][kJacThreads / 32];
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
    part[2 * blockIdx.x] = x;
    part[2 * blockIdx.x + 1] = y;
  }
}

// Every block sums the partial norms in the same order: same decision everywhere.
__device__ __forceinline__ bool decide_stop(const JacArgs& a, int sweep, double* thr) {
  __shared__ int s_stop;
  __shared__ double s_thr;
  if (threadIdx.x == 0) {
    double x = 0.0, y = 0.0;
    for (int b = 0; b < (int)gridDim.x; ++b) { x += a.part[2 * b]; y += a.part[2 * b + 1]; }
    int stop = (x <= a.tol * a.tol * y) || (y == 0.0);
    if (!stop && sweep >= a.max_sweeps) {
      flag_status(a.status, SKY_ENOCONV);
      stop = 1;
    }
    s_stop = stop;
    s_thr = 1e-19 * sqrt(y);     // rotations below this change nothing measurable
  }
  __syncthreads();
  *thr = s_thr;
  return s_stop != 0;
}

__global__ void __launch_bounds__(kJacThreads) k_jacobi(JacArgs a) {
  if (a.run && *a.run == 0) return;   // uniform across the grid: no barrier is entered
  const int m = a.m, n = a.n, h = m / 2;
  const int gtid = blockIdx.x * kJacThreads + threadIdx.x;
  const int gsz = gridDim.x * kJacThreads;
  double2* cur = a.A0;
  double2* nxt = a.A1;
  JRot* Rc = a.R0;
  JRot* Rn = a.R1;
  int which = 0;
  unsigned epoch = 0;
  // prologue: norms of the input
  {
    double off = 0.0, tot = 0.0;
    for (int e = gtid; e < n * n; e += gsz) {
      const int i = e / n, j = e % n;
      const double2 v = cur[(long long)i * m + j];
      const double w2 = v.x * v.x + v.y * v.y;
      tot += w2;
      if (i != j) off += w2;
    }
    block_norms(off, tot, a.part);
  }
  if (!grid_barrier(a.bar, epoch, a.status)) return;
  double thr;
  bool stop = decide_stop(a, 0, &thr);
  // rotations of round 0
  for (int k = gtid; k < h; k += gsz) {
    int p, q;
    pair_of(k, 0, m, p, q);
    Rc[k] = make_rot(cur[(long long)p * m + p].x, cur[(long long)q * m + q].x,
                     cur[(long long)p * m + q], p, q, n, thr);
  }
  if (!grid_barrier(a.bar, epoch, a.status)) return;
  const int nblk = h * h, nV = m * h;
  int sweeps_done = 0;
  for (int sweep = 1; !stop; ++sweep) {
    sweeps_done = sweep;
    for (int r = 0; r < m - 1; ++r) {
      const bool last = (r == m - 2);
      const int rn = last ? 0 : r + 1;
      double off = 0.0, tot = 0.0;
      // Pair indices follow from (k, r) alone, so every item issues its matrix
      // loads together with the rotation loads (one L2 round trip, not two).
      for (int w = gtid; w < nblk + nV + h; w += gsz) {
        if (w < nblk) {
          // 2x2 block (P1 rows, P2 columns): B' = J1^H B J2 into the other buffer
          const int k1 = w / h, k2 = w % h;
          int p1, q1, p2, q2;
          pair_of(k1, r, m, p1, q1);
          pair_of(k2, r, m, p2, q2);
          const long long i00 = (long long)p1 * m + p2, i01 = (long long)p1 * m + q2;
          const long long i10 = (long long)q1 * m + p2, i11 = (long long)q1 * m + q2;
          const double2 b00 = cur[i00], b01 = cur[i01], b10 = cur[i10], b11 = cur[i11];
          const JRot R1 = Rc[k1];
          const JRot R2 = Rc[k2];
          double2 o00, o01, o10, o11;
          if (R1.id && R2.id) {
            o00 = b00; o01 = b01; o10 = b10; o11 = b11;
          } else if (k1 == k2) {
            // pivot block: the exact result of the 2x2 diagonalisation
            o00 = make_double2(R1.dp, 0.0); o11 = make_double2(R1.dq, 0.0);
            o01 = make_double2(0.0, 0.0); o10 = o01;
          } else {
            double2 t0, t1;
            right_col(R2, 0, b00, b01, b10, b11, t0, t1);
            o00 = left_row(R1, 0, t0, t1);
            o10 = left_row(R1, 1, t0, t1);
            right_col(R2, 1, b00, b01, b10, b11, t0, t1);
            o01 = left_row(R1, 0, t0, t1);
            o11 = left_row(R1, 1, t0, t1);
          }
          nxt[i00] = o00; nxt[i01] = o01; nxt[i10] = o10; nxt[i11] = o11;
          if (last) {
            const double w00 = o00.x * o00.x + o00.y * o00.y, w01 = o01.x * o01.x + o01.y * o01.y;
            const double w10 = o10.x * o10.x + o10.y * o10.y, w11 = o11.x * o11.x + o11.y * o11.y;
            tot += w00 + w01 + w10 + w11;
            off += (p1 != p2 ? w00 : 0.0) + (p1 != q2 ? w01 : 0.0) +
                   (q1 != p2 ? w10 : 0.0) + (q1 != q2 ? w11 : 0.0);
          }
        } else if (w < nblk + nV) {
          // accumulate the rotation into row `row` of V (in place)
          const int u = w - nblk, row = u / h, k = u % h;
          int p, q;
          pair_of(k, r, m, p, q);
          double2* vr = a.V + (long long)row * m;
          const double2 vp = vr[p], vq = vr[q];
          const JRot R = Rc[k];
          if (!R.id) {
            vr[p] = rx_plus_cy(R.c, vp, R.j10, vq);
            vr[q] = rx_plus_cy(R.s, vp, R.j11, vq);
          }
        } else {
          // rotation of pair k of the next round from this round's result,
          // recomputed here from the old blocks (no extra barrier)
          const int k = w - nblk - nV;
          int p, q;
          pair_of(k, rn, m, p, q);
          const int kp = pair_index(p, r, m), kq = pair_index(q, r, m);
          int pp, pq, qp, qq;
          pair_of(kp, r, m, pp, pq);
          pair_of(kq, r, m, qp, qq);
          const double2 b00 = cur[(long long)pp * m + qp], b01 = cur[(long long)pp * m + qq];
          const double2 b10 = cur[(long long)pq * m + qp], b11 = cur[(long long)pq * m + qq];
          const double dpp = cur[(long long)p * m + p].x, dqq = cur[(long long)q * m + q].x;
          const JRot Rp = Rc[kp];
          const JRot Rq = Rc[kq];
          const int lp = (p == pp) ? 0 : 1, lq = (q == qp) ? 0 : 1;
          const double app = Rp.id ? dpp : (lp ? Rp.dq : Rp.dp);
          const double aqq = Rq.id ? dqq : (lq ? Rq.dq : Rq.dp);
          double2 t0, t1;
          right_col(Rq, lq, b00, b01, b10, b11, t0, t1);
          const double2 z = left_row(Rp, lp, t0, t1);
          Rn[k] = make_rot(app, aqq, z, p, q, n, thr);
        }
      }
      if (last) block_norms(off, tot, a.part);
      if (!grid_barrier(a.bar, epoch, a.status)) return;
      double2* tA = cur; cur = nxt; nxt = tA;
      JRot* tR = Rc; Rc = Rn; Rn = tR;
      which ^= 1;
    }
    stop = decide_stop(a, sweep, &thr);
    if (!stop) {
      // round-0 rotations were computed with the previous threshold; refresh
      // them with the new one (cheap; needs one barrier)
      for (int k = gtid; k < h; k += gsz) {
        int p, q;
        pair_of(k, 0, m, p, q);
        Rc[k] = make_rot(cur[(long long)p * m + p].x, cur[(long long)q * m + q].x,
                         cur[(long long)p * m + q], p, q, n, thr);
      }
      if (!grid_barrier(a.bar, epoch, a.status)) return;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *a.result = which;
    a.stats[0] += 1;
    a.stats[1] += sweeps_done;
    a.stats[2] = sweeps_done;
  }
}

// Copy A (n x n) into the padded m x m buffer, V = identity, reset the barrier.
__global__ void k_jacobi_init(const double2* A, int n, int m, double2* A0, double2* V,
                              unsigned* bar, int* result, const int* run) {
  if (run && *run == 0) return;
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e == 0) { bar[0] = 0u; *result = 0; }
  if (e >= (long long)m * m) return;
  const int i = (int)(e / m), j = (int)(e % m);
  A0[e] = (i < n && j < n) ? A[(long long)i * n + j] : make_double2(0.0, 0.0);
  V[e] = make_double2(i == j ? 1.0 : 0.0, 0.0);
}

// Eigenvalues ascending (ties by index) and the matching columns of V.
__global__ void k_jacobi_finish(const double2* A0, const double2* A1, const double2* V,
                                const int* result, int n, int m, double* w, double2* Z,
                                const int* run) {
  if (run && *run == 0) return;
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
  if (per_sm > 1) per_sm = 1;   // one block per SM keeps the barrier short
  return per_sm * c->num_sms;
}

size_t jacobi_rot_bytes(int m) { return (size_t)2 * (m / 2 + 1) * sizeof(JRot); }

sky_status eigh_impl(Ctx* c, const double2* A, int I, double* w, double2* Z, const int* run) {
  if (I == 0) return SKY_OK;
  const int m = I + (I & 1);
  k_jacobi_init<<<div_up((long long)m * m, 256), 256, 0, c->stream>>>(A, I, m, c->d_eigA[0],
                                                                      c->d_eigV, c->d_bar,
                                                                      c->d_eigres, run);
  note_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_check(c, e, "jacobi init");
  if (m >= 2) {
    const int h = m / 2;
    const long long items = (long long)h * h + (long long)m * h + h;
    int grid = (int)((items + kJacThreads - 1) / kJacThreads);
    if (grid < c->eig_grid / 2) grid = c->eig_grid / 2;   // spread the FP64 work over the SMs
    if (grid > c->eig_grid) grid = c->eig_grid;
    if (grid < 1) grid = 1;
    JacArgs a;
    a.A0 = c->d_eigA[0]; a.A1 = c->d_eigA[1]; a.V = c->d_eigV;
    a.R0 = reinterpret_cast<JRot*>(c->d_eigrot);
    a.R1 = a.R0 + h;
    a.n = I; a.m = m;
    a.tol = 1e-14;
    a.max_sweeps = 60;
    a.part = c->d_eigpart; a.bar = c->d_bar; a.status = c->d_status; a.result = c->d_eigres;
    a.run = run;
    a.stats = c->d_stats;
    void* args[] = {&a};
    note_launch();
    e = cudaLaunchCooperativeKernel((const void*)k_jacobi, dim3(grid), dim3(kJacThreads), args, 0,
                                    c->stream);
    if (e != cudaSuccess) return cuda_check(c, e, "jacobi");
  }
  k_jacobi_finish<<<div_up(I, 128), 128, 0, c->stream>>>(c->d_eigA[0], c->d_eigA[1], c->d_eigV,
                                                        c->d_eigres, I, m, w, Z, run);
  note_launch();
  return cuda_check(c, cudaGetLastError(), "jacobi finish");
}

// Y = X diag(lambda^{-1/2}); flags SKY_ENOTPD for a non-positive eigenvalue.
__global__ void k_inv_sqrt_cols(const double2* X, const double* lam, int n, double2* Y, int* status,
                                const int* run) {
  if (run && *run == 0) return;
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

// ---- Loewdin factor C = S^{-1/2} (Eq. Loewedin) ----------------------------
// C comes from the coupled Newton-Schulz iteration for the inverse square
// root (Higham, Functions of Matrices, 2008):  Y0 = S, Z0 = I;
// T = (3I - Z Y)/2;  Y <- Y T;  Z <- T Z;  then Z -> S^{-1/2}.  Eigenvalue by
// eigenvalue it is z <- z (3 - l z^2)/2 from z = 1, which converges to
// l^{-1/2} for 0 < l < 3 (quadratically once l z^2 is near 1).  It is used when
// the Gershgorin bound max_i sum_j |S_ij| is below kNsSwitch (|S_ij| bounded
// by |Re| + |Im|), which holds for the overlaps of damped orthonormal states.
// Otherwise, or if it has not converged after kNsMaxIter steps, C is
// X Lambda^{-1/2} X^H from the Jacobi eigendecomposition of S, as the paper
// describes.  Device gates: [0] Newton-Schulz running, [1] eigendecomposition
// needed, [2] Newton-Schulz converged (one final update pending or done),
// [3] Newton-Schulz chosen; [4..5] the row-sum bound as integer bits.
constexpr int kNsMaxIter = 14;
constexpr double kNsSwitch = 2.5;      // spectral bound for the Newton-Schulz route
constexpr double kNsConv = 1e-10;      // ||I - Z Y||_F after which one more update suffices

// Row sums of |S| (bounded by |Re| + |Im|) -> max into gate[4..5]; Y = S, Z = I.
__global__ void __launch_bounds__(256) k_ns_rows(const double2* S, int n, double2* Y, double2* Z,
                                                 int* gate) {
  __shared__ double red[8];
  const int i = blockIdx.x;
  double acc = 0.0;
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    const long long e = (long long)i * n + j;
    const double2 v = S[e];
    acc += fabs(v.x) + fabs(v.y);
    Y[e] = v;
    Z[e] = make_double2(i == j ? 1.0 : 0.0, 0.0);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    // non-negative doubles order like their bit patterns
    atomicMax(reinterpret_cast<unsigned long long*>(gate + 4),
              (unsigned long long)__double_as_longlong(t));
  }
}

__global__ void k_ns_reset(int* gate) {
  gate[0] = gate[1] = gate[2] = gate[3] = 0;
  *reinterpret_cast<unsigned long long*>(gate + 4) = 0ull;
}

__global__ void k_ns_choose(int* gate) {
  const double R = __longlong_as_double(*reinterpret_cast<long long*>(gate + 4));
  const int ns = R < kNsSwitch;
  gate[3] = ns;
  gate[0] = ns;
  gate[1] = !ns;
  gate[2] = 0;
}

// T = (3I - W)/2 in place of W = Z Y; records convergence; ends the
// iteration one step after convergence was seen.
__global__ void __launch_bounds__(1024) k_ns_step(double2* W, int n, int* gate, long long* stats) {
  __shared__ double red[32];
  __shared__ int s_skip;
  if (threadIdx.x == 0) {
    if (gate[0] && gate[2]) gate[0] = 0;   // the final update has been applied
    s_skip = !gate[0];
  }
  __syncthreads();
  if (s_skip) return;
  if (threadIdx.x == 0) stats[5] += 1;
  double acc = 0.0;
  for (long long e = threadIdx.x; e < (long long)n * n; e += blockDim.x) {
    const int i = (int)(e / n), j = (int)(e % n);
    double2 d = W[e];
    if (i == j) d.x -= 1.0;                 // W - I
    acc += d.x * d.x + d.y * d.y;
    W[e] = make_double2((i == j ? 1.0 : 0.0) - 0.5 * d.x, -0.5 * d.y);   // I - (W - I)/2
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    if (sqrt(t) < kNsConv) gate[2] = 1;
  }
}

__global__ void k_ns_copy(double2* Y, double2* Z, const double2* Yn, const double2* Zn, int n,
                          const int* gate) {
  if (!gate[0]) return;
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)n * n) return;
  Y[e] = Yn[e];
  Z[e] = Zn[e];
}

// C = (Z + Z^H)/2 when Newton-Schulz converged; otherwise request the
// eigendecomposition route.
__global__ void k_ns_final(const double2* Z, int n, double2* C, int* gate, long long* stats) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int ok = gate[3] && gate[2];
  if (e == 0) {
    stats[3] += 1;
    stats[4] += ok;
  }
  if (!ok) {
    if (e == 0) gate[1] = 1;
    return;
  }
  if (e >= (long long)n * n) return;
  const int i = (int)(e / n), j = (int)(e % n);
  C[e] = 0.5 * (Z[e] + conjx(Z[(long long)j * n + i]));
}

sky_status lowdin_impl(Ctx* c, const double2* S, int I, double2* C) {
  if (I == 0) return SKY_OK;
  double2 *Y = c->d_small[0], *Z = c->d_small[1], *W = c->d_small[2];
  double2 *Yn = c->d_small[3], *Zn = c->d_small[4];
  int* gate = c->d_gate;
  const long long nn = (long long)I * I;
  cudaError_t e;
  k_ns_reset<<<1, 1, 0, c->stream>>>(gate);
  k_ns_rows<<<I, 256, 0, c->stream>>>(S, I, Y, Z, gate);
  k_ns_choose<<<1, 1, 0, c->stream>>>(gate);
  note_launch(3);
  for (int it = 0; it < kNsMaxIter; ++it) {
    sky_status st = zgemm_small(c, false, false, Z, Y, W, I, gate, gate + 2);   // W = Z Y
    if (st != SKY_OK) return st;
    k_ns_step<<<1, 1024, 0, c->stream>>>(W, I, gate, c->d_stats);
    note_launch();
    st = zgemm_small(c, false, false, Y, W, Yn, I, gate);                       // Y T
    if (st == SKY_OK) st = zgemm_small(c, false, false, W, Z, Zn, I, gate);     // T Z
    if (st != SKY_OK) return st;
    k_ns_copy<<<div_up(nn, 256), 256, 0, c->stream>>>(Y, Z, Yn, Zn, I, gate);
    note_launch();
  }
  k_ns_final<<<div_up(nn, 256), 256, 0, c->stream>>>(Z, I, C, gate, c->d_stats);
  note_launch();
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_check(c, e, "newton-schulz");
  // eigendecomposition route (runs only when gate[1] is set)
  double2 *X = c->d_small[3], *Xs = c->d_small[4];
  sky_status st = eigh_impl(c, S, I, c->d_eigw, X, gate + 1);
  if (st != SKY_OK) return st;
  k_inv_sqrt_cols<<<div_up(nn, 256), 256, 0, c->stream>>>(X, c->d_eigw, I, Xs, c->d_status,
                                                          gate + 1);
  note_launch();
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_check(c, e, "loewdin scale");
  return zgemm_small(c, false, true, Xs, X, C, I, gate + 1);   // C = X Lambda^{-1/2} X^H
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
