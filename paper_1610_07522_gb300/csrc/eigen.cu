// FP64 Hermitian eigensolver for steps 3b-3c (Sec. 3.3.2) and the Loewdin /
// Rayleigh-Ritz factors built on it.
//
// The paper diagonalises with ScaLAPACK's tridiagonal + MRRR solver; its
// GPU counterpart is in eigen_tridiag.cu, and eigh_batch below picks between
// it and the solver of this file, a parallel cyclic Jacobi method (one launch
// for a whole batch of small problems): in each round the indices
// are paired by a round-robin tournament, every pair (p, q) gets the 2x2
// unitary J = D R (D removes the phase of A_pq, R is the real Jacobi
// rotation), and all (I/2)^2 2x2 blocks are updated at once as
// A'[P1,P2] = J1^H A[P1,P2] J2 (ping-pong buffers), with the rotations
// accumulated into V.  One sweep is I-1 rounds; sweeps stop when the
// off-diagonal Frobenius norm falls below tol * ||A||_F.  The whole solve is
// one cooperative kernel whose rounds are separated by a grid barrier with a
// bounded wait.  Near convergence the matrices are close to diagonal and a
// sweep or two suffices.
#include "eig_common.cuh"

namespace sky {

constexpr int kJacThreads = 512;

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

// ---- batched solve -----------------------------------------------------------
// Up to kMaxBatch independent Hermitian problems share one cooperative launch:
// every round serves all unfinished problems, so the fixed cost of a round
// (grid barrier, memory latency) is paid once for the batch.  Problem b works in
// its own slices of the workspace; its rounds follow its own size m_b.
struct JacProb {
  double2* A0; double2* A1; double2* V;
  JRot* R0; JRot* R1;   // rotations of the current / next round, [m/2] each
  int n, m;
};

struct JacBatch {
  JacProb p[kMaxBatch];
  // prefix offsets over problems of the three kinds of work items of a round:
  // next-round rotations (m/2), 2x2 block updates (h(h+1)/2), V row updates (m h)
  int offR[kMaxBatch + 1], offB[kMaxBatch + 1], offV[kMaxBatch + 1];
  int np;
  double tol;
  int max_sweeps;
  long long spins;      // spin budget of each grid-barrier wait
  double* part;         // [np][gridDim.x][2] partial norms
  unsigned* bar;
  int* status;
  int* result;          // [np] 0: A0 holds the result, 1: A1
  const int* run;       // problem b runs iff run == null or run[b * run_stride] != 0
  int run_stride;
  long long* stats;     // [0] solves, [1] sweeps in total, [2] sweeps of the last solve
};

// Per-block reduction of (off, tot) into part[2 * blockIdx.x] (blockDim == kJacThreads).
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
  __syncthreads();
}

// The same sums in every block, in the same order: the same decision everywhere.
__device__ __forceinline__ void sum_parts(const double* part, double& off, double& tot) {
  off = 0.0;
  tot = 0.0;
  for (int b = 0; b < (int)gridDim.x; ++b) { off += part[2 * b]; tot += part[2 * b + 1]; }
}

__global__ void __launch_bounds__(kJacThreads) k_jacobi(JacBatch a) {
  __shared__ int s_done[kMaxBatch], s_which[kMaxBatch], s_sweep[kMaxBatch];
  __shared__ double s_thr[kMaxBatch];
  __shared__ double s_acc[kMaxBatch][2];   // (off, tot) of problems ending a sweep
  const int gtid = blockIdx.x * kJacThreads + threadIdx.x;
  const int gsz = gridDim.x * kJacThreads;
  const int np = a.np;
  unsigned epoch = 0;
  // ---- prologue: norms of every problem (||A||_F is invariant under the rotations)
  for (int b = 0; b < np; ++b) {
    const JacProb& P = a.p[b];
    double off = 0.0, tot = 0.0;
    for (long long e = gtid; e < (long long)P.n * P.n; e += gsz) {
      const int i = (int)(e / P.n), j = (int)(e % P.n);
      const double2 v = P.A0[(long long)i * P.m + j];
      const double w2 = v.x * v.x + v.y * v.y;
      tot += w2;
      if (i != j) off += w2;
    }
    block_norms(off, tot, a.part + (long long)b * 2 * gridDim.x);
  }
  if (!grid_barrier(a.bar, epoch, a.status, a.spins)) return;
  // per-problem bookkeeping: thread b of every block serves problem b (the same
  // sums in the same order in every block, so every block decides alike)
  int act = 0;
  for (int b = threadIdx.x; b < np; b += blockDim.x) {
    double off, tot;
    sum_parts(a.part + (long long)b * 2 * gridDim.x, off, tot);
    const bool run = !a.run || a.run[b * a.run_stride] != 0;
    s_done[b] = !run || (off <= a.tol * a.tol * tot) || (tot == 0.0) || a.p[b].m < 2;
    s_thr[b] = 1e-19 * sqrt(tot);   // rotations below this change nothing measurable
    s_which[b] = 0;
    s_sweep[b] = 0;
    s_acc[b][0] = s_acc[b][1] = 0.0;
    act |= !s_done[b];
  }
  int active = __syncthreads_or(act);
  // rotations of round 0
  for (int b = 0; b < np; ++b) {
    if (s_done[b]) continue;
    const JacProb& P = a.p[b];
    const int h = P.m / 2;
    for (int k = gtid; k < h; k += gsz) {
      int p, q;
      pair_of(k, 0, P.m, p, q);
      P.R0[k] = make_rot(P.A0[(long long)p * P.m + p].x, P.A0[(long long)q * P.m + q].x,
                         P.A0[(long long)p * P.m + q], p, q, P.n, s_thr[b]);
    }
  }
  if (!grid_barrier(a.bar, epoch, a.status, a.spins)) return;
  for (int t = 0; active; ++t) {
    // One item per thread.  Work is dealt out in 32-item warp chunks round-robin
    // over the blocks, so every SM gets an even share of each kind of item (the
    // FP64 units of one SM are narrow) while warps keep contiguous items.
    // Items: next-round rotations, then 2x2 block updates, then V row updates.
    // Pair indices follow from (k, r) alone, so every item issues its matrix
    // loads together with the rotation loads (one L2 round trip).
    const int nR = a.offR[np], nB = a.offB[np], total = nR + nB + a.offV[np];
    const int lane = threadIdx.x & 31, wslot = threadIdx.x >> 5;
    const int nwarps = gridDim.x * (kJacThreads / 32);
    for (int ch = wslot * (int)gridDim.x + blockIdx.x; ch * 32 < total; ch += nwarps) {
      int w = ch * 32 + lane;
      if (w >= total) continue;
      if (w < nR) {
        // rotation of pair k of the next round from this round's result,
        // recomputed from the old blocks (no extra barrier)
        const int b = find_prob(a.offR, np, w);
        if (s_done[b]) continue;
        const JacProb& P = a.p[b];
        const int m = P.m, n = P.n;
        const int r = t % (m - 1);
        const int rn = (r == m - 2) ? 0 : r + 1;
        const double2* cur = s_which[b] ? P.A1 : P.A0;
        const JRot* Rc = (t & 1) ? P.R1 : P.R0;
        JRot* Rn = (t & 1) ? P.R0 : P.R1;
        const int k = w - a.offR[b];
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
        Rn[k] = make_rot(app, aqq, z, p, q, n, s_thr[b]);
      } else if ((w -= nR) < nB) {
        // 2x2 block (P1 rows, P2 columns), k1 >= k2: B' = J1^H B J2 into the
        // other buffer, and its conjugate transpose into the mirrored block
        const int b = find_prob(a.offB, np, w);
        if (s_done[b]) continue;
        const JacProb& P = a.p[b];
        const int m = P.m;
        const int r = t % (m - 1);
        const bool last = (r == m - 2);
        const double2* cur = s_which[b] ? P.A1 : P.A0;
        double2* nxt = s_which[b] ? P.A0 : P.A1;
        const JRot* Rc = (t & 1) ? P.R1 : P.R0;
        const int u = w - a.offB[b];
        int k1 = (int)((sqrtf(8.0f * (float)u + 1.0f) - 1.0f) * 0.5f);
        while ((k1 + 1) * (k1 + 2) / 2 <= u) ++k1;
        while (k1 * (k1 + 1) / 2 > u) --k1;
        const int k2 = u - k1 * (k1 + 1) / 2;
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
        if (k1 != k2) {
          nxt[(long long)p2 * m + p1] = conjx(o00);
          nxt[(long long)q2 * m + p1] = conjx(o01);
          nxt[(long long)p2 * m + q1] = conjx(o10);
          nxt[(long long)q2 * m + q1] = conjx(o11);
        }
        if (last) {
          const double w00 = o00.x * o00.x + o00.y * o00.y, w01 = o01.x * o01.x + o01.y * o01.y;
          const double w10 = o10.x * o10.x + o10.y * o10.y, w11 = o11.x * o11.x + o11.y * o11.y;
          const double mult = (k1 != k2) ? 2.0 : 1.0;   // the mirrored block counts too
          atomicAdd(&s_acc[b][1], mult * (w00 + w01 + w10 + w11));
          atomicAdd(&s_acc[b][0], mult * ((p1 != p2 ? w00 : 0.0) + (p1 != q2 ? w01 : 0.0) +
                                          (q1 != p2 ? w10 : 0.0) + (q1 != q2 ? w11 : 0.0)));
        }
      } else {
        w -= nB;
        // accumulate the rotation into row `row` of V (in place)
        const int b = find_prob(a.offV, np, w);
        if (s_done[b]) continue;
        const JacProb& P = a.p[b];
        const int m = P.m, h = m / 2;
        const int r = t % (m - 1);
        const JRot* Rc = (t & 1) ? P.R1 : P.R0;
        const int v = w - a.offV[b], row = v / h, k = v % h;
        int p, q;
        pair_of(k, r, m, p, q);
        double2* vr = P.V + (long long)row * m;
        const double2 vp = vr[p], vq = vr[q];
        const JRot R = Rc[k];
        if (!R.id) {
          vr[p] = rx_plus_cy(R.c, vp, R.j10, vq);
          vr[q] = rx_plus_cy(R.s, vp, R.j11, vq);
        }
      }
    }
    // partial norms of the problems that end a sweep this round
    __syncthreads();
    for (int b = threadIdx.x; b < np; b += blockDim.x) {
      if (s_done[b] || (t % (a.p[b].m - 1)) != a.p[b].m - 2) continue;
      double* part = a.part + (long long)b * 2 * gridDim.x;
      part[2 * blockIdx.x] = s_acc[b][0];
      part[2 * blockIdx.x + 1] = s_acc[b][1];
      s_acc[b][0] = s_acc[b][1] = 0.0;
    }
    if (!grid_barrier(a.bar, epoch, a.status, a.spins)) return;
    act = 0;
    for (int b = threadIdx.x; b < np; b += blockDim.x) {
      if (s_done[b]) continue;
      s_which[b] ^= 1;
      if ((t % (a.p[b].m - 1)) == a.p[b].m - 2) {
        s_sweep[b] += 1;
        double off, tot;
        sum_parts(a.part + (long long)b * 2 * gridDim.x, off, tot);
        if (off <= a.tol * a.tol * tot || tot == 0.0) {
          s_done[b] = 1;
        } else if (s_sweep[b] >= a.max_sweeps) {
          flag_status(a.status, SKY_ENOCONV);
          s_done[b] = 1;
        }
      }
      act |= !s_done[b];
    }
    active = __syncthreads_or(act);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    for (int b = 0; b < np; ++b) {
      a.result[b] = s_which[b];
      const bool run = !a.run || a.run[b * a.run_stride] != 0;
      if (run) {
        a.stats[0] += 1;
        a.stats[1] += s_sweep[b];
        a.stats[2] = s_sweep[b];
      }
    }
  }
}

struct EigJobs {
  const double2* A[kMaxBatch];
  double* w[kMaxBatch];
  double2* Z[kMaxBatch];
  double2* A0[kMaxBatch];
  double2* A1[kMaxBatch];
  double2* V[kMaxBatch];
  int n[kMaxBatch], m[kMaxBatch];
  int np;
  const int* run;
  int run_stride;
};

// Copy each A (n x n) into its padded m x m buffer, V = identity, reset the barrier.
__global__ void k_jacobi_init(EigJobs j, unsigned* bar, int* result) {
  const int b = blockIdx.y;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    result[b] = 0;
    if (b == 0) bar[0] = 0u;
  }
  if (j.run && j.run[b * j.run_stride] == 0) return;
  const int n = j.n[b], m = j.m[b];
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < (long long)m * m;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / m), k = (int)(e % m);
    j.A0[b][e] = (i < n && k < n) ? j.A[b][(long long)i * n + k] : make_double2(0.0, 0.0);
    j.V[b][e] = make_double2(i == k ? 1.0 : 0.0, 0.0);
  }
}

// Eigenvalues ascending (ties by index) and the matching columns of V.
__global__ void k_jacobi_finish(EigJobs j, const int* result) {
  const int b = blockIdx.y;
  if (j.run && j.run[b * j.run_stride] == 0) return;
  const int n = j.n[b], m = j.m[b];
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  const double2* A = result[b] ? j.A1[b] : j.A0[b];
  const double dc = A[(long long)c * m + c].x;
  int rank = 0;
  for (int i = 0; i < n; ++i) {
    const double di = A[(long long)i * m + i].x;
    rank += (di < dc) || (di == dc && i < c);
  }
  j.w[b][rank] = dc;
  for (int i = 0; i < n; ++i) j.Z[b][(long long)i * n + rank] = j.V[b][(long long)i * m + c];
}

constexpr int kJacobiLarge = 512;   // problem size from which the untuned Jacobi uses 2 blocks/SM

int jacobi_max_grid(Ctx* c) {
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_jacobi, kJacThreads, 0);
  if (per_sm < 1) per_sm = 1;
  if (per_sm > 2) per_sm = 2;   // the tunable maximum; the default is one block per SM
  return per_sm * c->num_sms;
}

size_t jacobi_rot_bytes(int m) { return (size_t)2 * (m / 2 + 1) * sizeof(JRot); }

// Jacobi eigendecomposition of np Hermitian matrices A[b] (n[b] x n[b]) into
// ascending w[b] and eigenvector columns Z[b]; problem b is skipped when
// run[b*stride] == 0.
static sky_status eigh_batch_jacobi(Ctx* c, int np, const double2* const* A, const int* n,
                                    double* const* w, double2* const* Z, const int* run,
                                    int run_stride) {
  EigJobs j;
  JacBatch a;
  long long items = 0;
  int nmax = 1, mmax = 2;
  j.np = np; j.run = run; j.run_stride = run_stride;
  a.np = np; a.offR[0] = a.offB[0] = a.offV[0] = 0;
  for (int b = 0; b < np; ++b) {
    const int m = n[b] + (n[b] & 1);
    const int h = m / 2;
    double2* base = c->d_eigA[0] + (size_t)b * c->eig_slot;
    j.A[b] = A[b]; j.w[b] = w[b]; j.Z[b] = Z[b]; j.n[b] = n[b]; j.m[b] = m;
    j.A0[b] = base;
    j.A1[b] = c->d_eigA[1] + (size_t)b * c->eig_slot;
    j.V[b] = c->d_eigV + (size_t)b * c->eig_slot;
    JacProb& P = a.p[b];
    P.A0 = j.A0[b]; P.A1 = j.A1[b]; P.V = j.V[b];
    P.R0 = reinterpret_cast<JRot*>(c->d_eigrot) + (size_t)b * 2 * (c->eig_slot_rot);
    P.R1 = P.R0 + c->eig_slot_rot;
    P.n = n[b]; P.m = m;
    items += (long long)h * (h + 1) / 2 + (long long)m * h + h;
    a.offR[b + 1] = a.offR[b] + h;
    a.offB[b + 1] = a.offB[b] + h * (h + 1) / 2;
    a.offV[b + 1] = a.offV[b] + m * h;
    if (n[b] > nmax) nmax = n[b];
    if (m > mmax) mmax = m;
  }
  cudaError_t e;
  dim3 gi(div_up((long long)mmax * mmax, 256) < 1024 ? div_up((long long)mmax * mmax, 256) : 1024, np);
  k_jacobi_init<<<gi, 256, 0, c->stream>>>(j, c->d_bar, c->d_eigres);
  note_launch();
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_check(c, e, "jacobi init");
  (void)items;
  // every SM's FP64 units share each round; until tuned, two blocks per SM for
  // large problems (FP64 bound: more warps hide latency) and one for small ones
  // (barrier bound: fewer blocks make the barrier cheaper), measured on GB300
  int grid = c->eig_grid;
  if (c->eig_grid_auto && nmax >= kJacobiLarge) grid = c->eig_grid_max;
  a.tol = 1e-14;
  a.max_sweeps = c->jac_max_sweeps;
  a.spins = c->wait_spins;
  a.part = c->d_eigpart; a.bar = c->d_bar; a.status = c->d_status; a.result = c->d_eigres;
  a.run = run; a.run_stride = run_stride;
  a.stats = c->d_stats;
  void* args[] = {&a};
  note_launch();
  e = cudaLaunchCooperativeKernel((const void*)k_jacobi, dim3(grid), dim3(kJacThreads), args, 0,
                                  c->stream);
  if (e != cudaSuccess) return cuda_check(c, e, "jacobi");
  k_jacobi_finish<<<dim3(div_up(nmax, 128), np), 128, 0, c->stream>>>(j, c->d_eigres);
  note_launch();
  return cuda_check(c, cudaGetLastError(), "jacobi finish");
}

// Until the method is set, batches with a problem of kTriAutoMin states or more
// take the tridiagonal route (O(n^3) once instead of per Jacobi sweep; a batch
// of many problems splits its blocks into teams); batches of small problems
// only stay with the batched Jacobi solver, whose rounds serve the whole
// batch at once.
constexpr int kTriAutoMin = 64;

// Eigendecomposition of np Hermitian matrices A[b] (n[b] x n[b]) into ascending
// w[b] and eigenvector columns Z[b]; problem b is skipped when run[b*stride] == 0.
sky_status eigh_batch(Ctx* c, int np, const double2* const* A, const int* n, double* const* w,
                      double2* const* Z, const int* run, int run_stride) {
  if (np < 1) return SKY_OK;
  if (np > c->eig_batch) return set_err(c, SKY_EINVAL, "eigensolver batch %d > %d", np, c->eig_batch);
  int nmax = 0;
  for (int b = 0; b < np; ++b) nmax = n[b] > nmax ? n[b] : nmax;
  const bool tri = c->eig_method == SKY_EIG_TRIDIAGONAL ||
                   (c->eig_method == SKY_EIG_AUTO && nmax >= kTriAutoMin);
  if (tri) {
    const sky_status s = eigh_batch_tri(c, np, A, n, w, Z, run, run_stride);
    if (s != SKY_EUNSUPPORTED) return s;
  }
  return eigh_batch_jacobi(c, np, A, n, w, Z, run, run_stride);
}

sky_status eigh_impl(Ctx* c, const double2* A, int I, double* w, double2* Z, const int* run) {
  if (I == 0) return SKY_OK;
  return eigh_batch(c, 1, &A, &I, &w, &Z, run, 0);
}

// Y = X diag(lambda^{-1/2}); flags SKY_ENOTPD for a non-positive eigenvalue.
struct ScaleJobs {
  const double2* X[kMaxBatch];
  const double* lam[kMaxBatch];
  double2* Y[kMaxBatch];
  int n[kMaxBatch];
};
__global__ void k_inv_sqrt_cols(ScaleJobs j, int* status, const int* run, int run_stride) {
  const int b = blockIdx.y;
  if (run && run[b * run_stride] == 0) return;
  const int n = j.n[b];
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)n * n) return;
  const int c = (int)(e % n);
  double l = j.lam[b][c];
  if (!(l > 0.0)) {
    if (e == c) flag_status(status, SKY_ENOTPD);
    l = 1e-300;
  }
  j.Y[b][e] = (1.0 / sqrt(l)) * j.X[b][e];
}

// H' = (H' + H'^H) / 2 in place.
struct HermJobs {
  double2* A[kMaxBatch];
  int n[kMaxBatch];
};
__global__ void k_hermitize(HermJobs h) {
  const int b = blockIdx.y;
  double2* A = h.A[b];
  const int n = h.n[b];
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)n * n) return;
  const int i = (int)(e / n), k = (int)(e % n);
  if (i > k) return;
  const double2 x = A[(long long)i * n + k], y = A[(long long)k * n + i];
  const double2 s = 0.5 * (x + conjx(y));
  A[(long long)i * n + k] = s;
  A[(long long)k * n + i] = conjx(s);
}

// ---- Loewdin factor C = S^{-1/2} (Eq. Loewedin) ----------------------------
// C comes from the coupled Newton-Schulz iteration for the inverse square
// root (Higham, Functions of Matrices, 2008):  Y0 = S, Z0 = I;
// T = (3I - Z Y)/2;  Y <- Y T;  Z <- T Z;  then Z -> S^{-1/2}.  Eigenvalue by
// eigenvalue it is z <- z (3 - l z^2)/2 from z = 1, which converges to
// l^{-1/2} for 0 < l < 3 (quadratically once l z^2 is near 1).  It is used when
// the Gershgorin bound max_i sum_j |S_ij| is below kNsSwitch (|S_ij| bounded
// by |Re| + |Im|) or when ||S - I||_F < kNsFrob (then every eigenvalue lies
// within kNsFrob of 1); one of them holds for the overlaps of damped
// orthonormal states, the Frobenius test being the sharper one at large I.
// Otherwise, or if it has not converged after kNsMaxIter steps, C is
// X Lambda^{-1/2} X^H from the Jacobi eigendecomposition of S, as the paper
// describes.  Device gates per problem b at gate[8 b + k]: [0] Newton-Schulz
// running, [1] eigendecomposition needed, [2] Newton-Schulz converged (one
// final update pending or done), [3] Newton-Schulz chosen; [4..5] the row-sum
// bound as integer bits; [6..7] ||S - I||_F^2 as a double.
constexpr int kNsMaxIter = 14;
constexpr double kNsSwitch = 2.5;      // spectral bound for the Newton-Schulz route
constexpr double kNsFrob = 0.9;        // ||S - I||_F bound for the same route
constexpr double kNsConv = 1e-7;       // ||I - Z Y||_F after which one more update suffices
                                       // (it squares the residual: ~1e-14)

struct NsJobs {
  const double2* S[kMaxBatch];
  double2* Y[kMaxBatch];
  double2* Z[kMaxBatch];
  double2* W[kMaxBatch];
  double2* Yn[kMaxBatch];
  double2* Zn[kMaxBatch];
  double2* C[kMaxBatch];
  int n[kMaxBatch];
};

__global__ void k_ns_reset(int* gate) {
  int* g = gate + 8 * threadIdx.x;
  g[0] = g[1] = g[2] = g[3] = 0;
  *reinterpret_cast<unsigned long long*>(g + 4) = 0ull;
  *reinterpret_cast<double*>(g + 6) = 0.0;
}

// Row sums of |S| (bounded by |Re| + |Im|) -> max into gate[4..5];
// sum of |S - I|^2 -> gate[6..7]; Y = S, Z = I.
__global__ void __launch_bounds__(256) k_ns_rows(NsJobs j, int* gate) {
  __shared__ double red[8], red2[8];
  const int b = blockIdx.y, n = j.n[b], i = blockIdx.x;
  if (i >= n) return;
  double acc = 0.0, fro = 0.0;
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    const long long e = (long long)i * n + k;
    const double2 v = j.S[b][e];
    acc += fabs(v.x) + fabs(v.y);
    const double dr = v.x - (i == k ? 1.0 : 0.0);
    fro += dr * dr + v.y * v.y;
    j.Y[b][e] = v;
    j.Z[b][e] = make_double2(i == k ? 1.0 : 0.0, 0.0);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    acc += __shfl_down_sync(0xffffffffu, acc, o);
    fro += __shfl_down_sync(0xffffffffu, fro, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[threadIdx.x >> 5] = acc;
    red2[threadIdx.x >> 5] = fro;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0, f = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { t += red[w]; f += red2[w]; }
    // non-negative doubles order like their bit patterns
    atomicMax(reinterpret_cast<unsigned long long*>(gate + 8 * b + 4),
              (unsigned long long)__double_as_longlong(t));
    atomicAdd(reinterpret_cast<double*>(gate + 8 * b + 6), f);
  }
}

__global__ void k_ns_choose(int* gate) {
  int* g = gate + 8 * threadIdx.x;
  const double R = __longlong_as_double(*reinterpret_cast<long long*>(g + 4));
  const double F = *reinterpret_cast<const double*>(g + 6);
  const int ns = R < kNsSwitch || F < kNsFrob * kNsFrob;
  g[3] = ns;
  g[0] = ns;
  g[1] = !ns;
  g[2] = 0;
}

// T = (3I - W)/2 in place of W = Z Y; records convergence; ends the
// iteration one step after convergence was seen.  Block b serves problem b.
__global__ void __launch_bounds__(1024) k_ns_step(NsJobs j, int* gate, long long* stats) {
  __shared__ double red[32];
  __shared__ int s_skip;
  const int b = blockIdx.x, n = j.n[b];
  int* g = gate + 8 * b;
  if (threadIdx.x == 0) {
    if (g[0] && g[2]) g[0] = 0;   // the final update has been applied
    s_skip = !g[0];
  }
  __syncthreads();
  if (s_skip) return;
  if (threadIdx.x == 0) atomicAdd(reinterpret_cast<unsigned long long*>(stats + 5), 1ull);
  double2* W = j.W[b];
  double acc = 0.0;
  for (long long e = threadIdx.x; e < (long long)n * n; e += blockDim.x) {
    const int i = (int)(e / n), k = (int)(e % n);
    double2 d = W[e];
    if (i == k) d.x -= 1.0;                 // W - I
    acc += d.x * d.x + d.y * d.y;
    W[e] = make_double2((i == k ? 1.0 : 0.0) - 0.5 * d.x, -0.5 * d.y);   // I - (W - I)/2
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    if (sqrt(t) < kNsConv) g[2] = 1;
  }
}

__global__ void k_ns_copy(NsJobs j, const int* gate) {
  const int b = blockIdx.y, n = j.n[b];
  if (!gate[8 * b]) return;
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)n * n) return;
  j.Y[b][e] = j.Yn[b][e];
  j.Z[b][e] = j.Zn[b][e];
}

// C = (Z + Z^H)/2 when Newton-Schulz converged; otherwise request the
// eigendecomposition route.
__global__ void k_ns_final(NsJobs j, int* gate, long long* stats) {
  const int b = blockIdx.y, n = j.n[b];
  int* g = gate + 8 * b;
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int ok = g[3] && g[2];
  if (e == 0) {
    atomicAdd(reinterpret_cast<unsigned long long*>(stats + 3), 1ull);
    atomicAdd(reinterpret_cast<unsigned long long*>(stats + 4), (unsigned long long)ok);
  }
  if (!ok) {
    if (e == 0) g[1] = 1;
    return;
  }
  if (e >= (long long)n * n) return;
  const int i = (int)(e / n), k = (int)(e % n);
  j.C[b][e] = 0.5 * (j.Z[b][e] + conjx(j.Z[b][(long long)k * n + i]));
}

sky_status lowdin_batch(Ctx* c, int np, const double2* const* S, const int* I, double2* const* C) {
  if (np < 1) return SKY_OK;
  if (np > c->eig_batch) return set_err(c, SKY_EINVAL, "Loewdin batch %d > %d", np, c->eig_batch);
  NsJobs j;
  int nmax = 1;
  for (int b = 0; b < np; ++b) {
    const size_t off = (size_t)b * c->small_slot;
    j.S[b] = S[b]; j.n[b] = I[b]; j.C[b] = C[b];
    j.Y[b] = c->d_small[0] + off; j.Z[b] = c->d_small[1] + off; j.W[b] = c->d_small[2] + off;
    j.Yn[b] = c->d_small[3] + off; j.Zn[b] = c->d_small[4] + off;
    if (I[b] > nmax) nmax = I[b];
  }
  int* gate = c->d_gate;
  const long long nn = (long long)nmax * nmax;
  cudaError_t e;
  k_ns_reset<<<1, np, 0, c->stream>>>(gate);
  k_ns_rows<<<dim3(nmax, np), 256, 0, c->stream>>>(j, gate);
  k_ns_choose<<<1, np, 0, c->stream>>>(gate);
  note_launch(3);
  const int *run[kMaxBatch], *stop[kMaxBatch], *fb[kMaxBatch];
  for (int b = 0; b < np; ++b) {
    run[b] = gate + 8 * b;
    stop[b] = gate + 8 * b + 2;
    fb[b] = gate + 8 * b + 1;
  }
  const int* none[kMaxBatch] = {nullptr};
  for (int it = 0; it < kNsMaxIter; ++it) {
    ZJobs w_ = zjobs(np, false, false, (const double2* const*)j.Z, (const double2* const*)j.Y, j.W, I, run, stop);
    sky_status st = zgemm_batch(c, w_);   // W = Z Y
    if (st != SKY_OK) return st;
    k_ns_step<<<np, 1024, 0, c->stream>>>(j, gate, c->d_stats);
    note_launch();
    ZJobs y_ = zjobs(np, false, false, (const double2* const*)j.Y, (const double2* const*)j.W, j.Yn, I, run, none);
    ZJobs z_ = zjobs(np, false, false, (const double2* const*)j.W, (const double2* const*)j.Z, j.Zn, I, run, none);
    if ((st = zgemm_batch(c, y_)) != SKY_OK) return st;                      // Y T
    if ((st = zgemm_batch(c, z_)) != SKY_OK) return st;                      // T Z
    k_ns_copy<<<dim3(div_up(nn, 256), np), 256, 0, c->stream>>>(j, gate);
    note_launch();
  }
  k_ns_final<<<dim3(div_up(nn, 256), np), 256, 0, c->stream>>>(j, gate, c->d_stats);
  note_launch();
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_check(c, e, "newton-schulz");
  // eigendecomposition route (problem b runs only when gate[8 b + 1] is set)
  double2* X[kMaxBatch];
  double* lam[kMaxBatch];
  ScaleJobs sj;
  for (int b = 0; b < np; ++b) {
    const size_t off = (size_t)b * c->small_slot;
    X[b] = c->d_small[3] + off;
    lam[b] = c->d_eigw + (size_t)b * (c->eig_slot_rot * 2 + 2);
    sj.X[b] = X[b]; sj.lam[b] = lam[b]; sj.Y[b] = c->d_small[4] + off; sj.n[b] = I[b];
  }
  sky_status st = eigh_batch(c, np, S, I, lam, X, gate + 1, 8);
  if (st != SKY_OK) return st;
  k_inv_sqrt_cols<<<dim3(div_up(nn, 256), np), 256, 0, c->stream>>>(sj, c->d_status, gate + 1, 8);
  note_launch();
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_check(c, e, "loewdin scale");
  ZJobs c_ = zjobs(np, false, true, (const double2* const*)sj.Y, (const double2* const*)X, C, I, fb, none);
  return zgemm_batch(c, c_);   // C = X Lambda^{-1/2} X^H
}

sky_status lowdin_impl(Ctx* c, const double2* S, int I, double2* C) {
  if (I == 0) return SKY_OK;
  return lowdin_batch(c, 1, &S, &I, &C);
}

// Rayleigh-Ritz for np problems: H' = C^H H C, H' = Z Lambda Z^H, M = C Z.
sky_status subspace_batch(Ctx* c, int np, const double2* const* H, const double2* const* C,
                          const int* I, double2* const* M, double* const* eps) {
  if (np < 1) return SKY_OK;
  if (np > c->eig_batch) return set_err(c, SKY_EINVAL, "subspace batch %d > %d", np, c->eig_batch);
  double2 *T1[kMaxBatch], *Hp[kMaxBatch], *Z[kMaxBatch];
  int nmax = 1;
  for (int b = 0; b < np; ++b) {
    const size_t off = (size_t)b * c->small_slot;
    T1[b] = c->d_small[0] + off; Hp[b] = c->d_small[1] + off; Z[b] = c->d_small[2] + off;
    if (I[b] > nmax) nmax = I[b];
  }
  const int* none[kMaxBatch] = {nullptr};
  sky_status st = zgemm_batch(c, zjobs(np, true, false, C, H, T1, I, none, none));   // C^H H
  if (st == SKY_OK)
    st = zgemm_batch(c, zjobs(np, false, false, (const double2* const*)T1, C, Hp, I, none, none));
  if (st != SKY_OK) return st;
  HermJobs hj;
  for (int b = 0; b < np; ++b) { hj.A[b] = Hp[b]; hj.n[b] = I[b]; }
  k_hermitize<<<dim3(div_up((long long)nmax * nmax, 256), np), 256, 0, c->stream>>>(hj);
  note_launch();
  cudaError_t e;
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_check(c, e, "hermitize");
  st = eigh_batch(c, np, (const double2* const*)Hp, I, eps, Z, nullptr, 0);
  if (st != SKY_OK) return st;
  return zgemm_batch(c, zjobs(np, false, false, C, (const double2* const*)Z, M, I, none, none));   // M = C Z
}

// Phase convention of the combined form: column k of Z is multiplied by the
// phase that makes its first component of largest modulus real and positive.
struct PhaseJobs {
  double2* Z[kMaxBatch];
  int n[kMaxBatch];
};
__global__ void k_fix_phase(PhaseJobs j) {
  const int b = blockIdx.y, n = j.n[b];
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  double2* Z = j.Z[b];
  int imax = 0;
  double amax = -1.0;
  for (int i = 0; i < n; ++i) {
    const double2 v = Z[(long long)i * n + k];
    const double a = v.x * v.x + v.y * v.y;
    if (a > amax) { amax = a; imax = i; }
  }
  const double2 z = Z[(long long)imax * n + k];
  const double r = sqrt(z.x * z.x + z.y * z.y);
  const double2 ph = make_double2(z.x / r, -z.y / r);   // conj(z) / |z|
  for (int i = 0; i < n; ++i) {
    const long long e = (long long)i * n + k;
    Z[e] = cmul(Z[e], ph);
  }
}

// The paper's combined form (Sec. 3.3.3): Z from H itself (the non-orthonormal
// basis, phases as above), M = Z C, eps = the eigenvalues of H.
sky_status subspace_literal_batch(Ctx* c, int np, const double2* const* H,
                                  const double2* const* C, const int* I, double2* const* M,
                                  double* const* eps) {
  if (np < 1) return SKY_OK;
  if (np > c->eig_batch) return set_err(c, SKY_EINVAL, "subspace batch %d > %d", np, c->eig_batch);
  double2* Z[kMaxBatch];
  for (int b = 0; b < np; ++b) Z[b] = c->d_small[2] + (size_t)b * c->small_slot;
  const int* none[kMaxBatch] = {nullptr};
  sky_status st = eigh_batch(c, np, H, I, eps, Z, nullptr, 0);
  if (st != SKY_OK) return st;
  PhaseJobs pj;
  int nmax = 1;
  for (int b = 0; b < np; ++b) {
    pj.Z[b] = Z[b];
    pj.n[b] = I[b];
    if (I[b] > nmax) nmax = I[b];
  }
  k_fix_phase<<<dim3(div_up(nmax, 128), np), 128, 0, c->stream>>>(pj);
  note_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_check(c, e, "fix phase");
  return zgemm_batch(c, zjobs(np, false, false, (const double2* const*)Z, C, M, I, none, none));
}

sky_status subspace_impl(Ctx* c, const double2* H, const double2* C, int I, double2* M,
                         double* eps) {
  if (I == 0) return SKY_OK;
  return subspace_batch(c, 1, &H, &C, &I, &M, &eps);
}

}  // namespace sky
