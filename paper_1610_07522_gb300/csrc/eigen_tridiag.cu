// FP64 Hermitian eigensolver by reduction to real tridiagonal form, for the
// diagonalisations of steps 3b-3c (Sec. 3.3.2) at the sizes where the cyclic
// Jacobi method's O(I^3) work per sweep dominates an iteration.
//
// The paper hands these to ScaLAPACK's Hermitian tridiagonal reduction with
// the MRRR tridiagonal solver.  Here the same three stages are GPU kernels:
//
//  1. k_hh_tridiag: A = Q T Q^H with Q = H_0 H_1 ... H_{n-2}, each reflector
//     H_t = I - tau_t v_t v_t^H chosen so that H_t^H maps column t below the
//     diagonal onto beta_t e_1 with beta_t real (T is real symmetric).  One
//     cooperative kernel: the blocks keep the columns of the (full, Hermitian)
//     trailing matrix cyclically in shared memory.  The update by H_t is
//     A <- A - v w^H - w v^H with p = A v, w = tau p - (|tau|^2 v^H p / 2) v.
//     Each owner forms p_j = col_j^H v_t for its own columns, fused with that
//     column's update by the previous reflector, and publishes p, the next
//     column and its block's partial of v^H p; after one grid barrier every
//     block recomputes the next column and reflector itself (the same
//     arithmetic in every block), so each step costs one barrier.  The heads
//     of up to four problems run side by side on separate warp groups.
//  2. k_tri_bisect: eigenvalues of T by multisection on the count of
//     negative LDL^T pivots of T - x I, one warp (kBisLanes points) per
//     eigenvalue and round: FP32 counts first, then double-float ones (the
//     chip's FP64 latency makes an FP64 count ~10 times slower).
//  3. k_tri_vectors: eigenvectors of T by inverse iteration (Gaussian
//     elimination with partial pivoting of T - lambda I, factored once, then
//     kInvIters solves from a counter-based random start); eigenvalues closer
//     than kTightRel ||T|| are handled by one thread in order, each new vector
//     orthogonalised against the cluster's earlier ones after every solve (as
//     LAPACK's dstein does).  k_tri_window then applies first-order Loewdin
//     steps Y <- Y (3 I - Y^T Y) / 2, with Y^T Y formed only between
//     eigenvalues within kWinRel ||T|| of each other (the inverse-iteration
//     vectors' mutual overlaps fall off like eps ||T|| / gap).  k_hh_back
//     forms Z = Q Y, one warp per column, the reflectors applied in reverse
//     order.
//
// Eigenvalues come out ascending, eigenvectors as the columns of Z.
#include <algorithm>
#include <cmath>

#include "dd.cuh"
#include "eig_common.cuh"

namespace sky {

constexpr int kTriThreads = 512;
constexpr int kTriWarps = kTriThreads / 32;
constexpr int kBisLanes = 32;           // bisection points per eigenvalue and round: one warp,
                                        // so every eigenvalue has its own warp (one wave)
constexpr int kBisMaxRounds = 96;       // ample for 2 eps ||T|| at 33x per round
constexpr int kInvIters = 3;            // inverse-iteration solves per vector
constexpr int kVecThreads = 8;          // eigenvectors per block of k_tri_vectors
constexpr double kTightRel = 1e-9;      // cluster threshold relative to ||T||
constexpr double kWinRel = 0.05;        // Loewdin window relative to ||T||
constexpr int kWinMax = 128;            // neighbours per side in the window at most
constexpr int kWinThreads = 128;
constexpr int kWinChunks = (2 * kWinMax + 1 + 31) / 32;
constexpr int kBackWarps = 16;
constexpr size_t kTriSmemMax = 200 * 1024;   // dynamic shared memory of k_hh_tridiag / k_hh_back
constexpr double kEps = 2.220446049250313e-16;
constexpr int kTeamBarStride = 32;     // unsigned between team barrier counters (128 bytes)

struct TriBatch {
  const double2* A[kMaxBatch];   // input matrices, row-major n x n
  double* w[kMaxBatch];          // eigenvalues out (ascending)
  double2* Z[kMaxBatch];         // eigenvectors out, Z[i * n + k] = component i of vector k
  int n[kMaxBatch];
  int rot[kMaxBatch];            // column j of problem b lives in block (j + rot) mod G
  int soff[kMaxBatch];           // own columns' offset in dynamic shared memory, -1: global
  int voff[kMaxBatch];           // offset of the block's three work vectors, -1: global
  double2* gvec;                 // per (problem slot, block) work vectors when voff = -1
  size_t gvec_stride;            // double2 per (problem slot, block) in gvec
  int coff;                      // offset of the per-column partials (doubles) in shared memory
  int off[kMaxBatch + 1];        // prefix sums of n: eigenvalue / column items
  int sid[kMaxBatch];            // workspace slot of each problem
  int np;
  double2* S0;                   // per problem: own columns (global home), later U0, U1
  double2* S1;                   // per problem: reflectors V[t * n + i]
  double2* S2;                   // per problem: Y and its Loewdin ping-pong buffer
  size_t slot;                   // double2 per problem in S0, S1, S2
  double* T;                     // per problem: U2, published vectors, tau, d, e, e^2, lambda
  size_t tslot;                  // doubles per problem in T
  int m;                         // stride of the vectors in T (even, >= every n)
  const int* run;                // problem b runs iff run == null or run[b * run_stride] != 0
  int run_stride;
  double* sp;                    // per problem slot: [2][gridDim.x] partials of Re(v^H p)
  size_t sp_stride;
  unsigned* bar;
  int* status;
  long long spins;
  long long* stats;
  // Teams (stage 1): the blocks tg0[k] .. tg0[k+1]-1 reduce the problems
  // tmem[tp0[k]] .. tmem[tp0[k+1]-1] by themselves, with their own barrier
  // counter tbar[kTeamBarStride k]; one team of all blocks when nteam = 1.
  int nteam;
  int tmem[kMaxBatch];
  int tp0[kMaxBatch + 1];
  int tg0[kMaxBatch + 1];
  unsigned* tbar;
};

// This block's team: its size G, the block's rank gb in it, its problems
// (positions p0 .. p1-1 of tmem) and its barrier counter.
struct TeamView {
  int G, gb, p0, p1;
  unsigned* bar;
};

struct TriPtrs {
  double2* cols;                 // own columns, global home: column j at cols + j * n
  double2* V;
  double *Y, *Y2, *U0, *U1, *U2;
  double2 *P0, *P1, *C0, *C1, *tau;
  double *d, *e, *e2, *lam;
  float *df, *e2f;               // d and e^2 rounded to float (coarse bisection rounds)
  dd *ddd, *e2dd;                // d and e^2 as float pairs (fine bisection rounds)
};

__device__ __forceinline__ TriPtrs tri_ptrs(const TriBatch& a, int b) {
  TriPtrs p;
  const size_t n = (size_t)a.n[b], m = (size_t)a.m, k = (size_t)a.sid[b];
  p.cols = a.S0 + k * a.slot;
  p.U0 = reinterpret_cast<double*>(p.cols);
  p.U1 = p.U0 + n * n;
  p.V = a.S1 + k * a.slot;
  p.Y = reinterpret_cast<double*>(a.S2 + k * a.slot);
  p.Y2 = p.Y + n * n;
  double* t = a.T + k * a.tslot;
  p.U2 = t;
  double2* vecs = reinterpret_cast<double2*>(t + m * m);   // m even: 16-byte aligned
  p.P0 = vecs; p.P1 = vecs + m; p.C0 = vecs + 2 * m; p.C1 = vecs + 3 * m; p.tau = vecs + 4 * m;
  double* s = reinterpret_cast<double*>(vecs + 5 * m);
  p.d = s; p.e = s + m; p.e2 = s + 2 * m; p.lam = s + 3 * m;
  p.ddd = reinterpret_cast<dd*>(s + 4 * m); p.e2dd = p.ddd + m;        // m doubles each
  p.df = reinterpret_cast<float*>(s + 6 * m); p.e2f = p.df + m;        // m / 2 doubles each
  return p;
}

// The block's three work vectors of problem b (v_t, v_{t-1}, w): in shared
// memory, or, for problems too large for it, a private copy per block in
// global memory (every block computes the same vectors itself, so the copies
// must not be shared between blocks).
__device__ __forceinline__ double2* vec_base(const TriBatch& a, int b, double2* dsm) {
  return a.voff[b] >= 0
             ? dsm + a.voff[b]
             : a.gvec + ((size_t)a.sid[b] * gridDim.x + blockIdx.x) * a.gvec_stride;
}

__device__ __forceinline__ bool tri_run(const TriBatch& a, int b) {
  return a.n[b] > 0 && (!a.run || a.run[b * a.run_stride] != 0);
}

// Warp sum by butterfly: every lane ends with the same total.
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ---- stage 1: Householder reduction ------------------------------------------
// The per-step vectors of a problem are short (n - t entries): its head work
// runs on one group of kHeadWarps warps, and the heads of up to kHeadGroups
// problems run side by side (one set of __syncthreads for all of them).
constexpr int kHeadWarps = 4;
constexpr int kHeadThreads = kHeadWarps * 32;
constexpr int kHeadGroups = kTriWarps / kHeadWarps;

__device__ __forceinline__ TeamView team_view(const TriBatch& a) {
  const int k = find_prob(a.tg0, a.nteam, (int)blockIdx.x);
  TeamView v;
  v.G = a.tg0[k + 1] - a.tg0[k];
  v.gb = (int)blockIdx.x - a.tg0[k];
  v.p0 = a.tp0[k];
  v.p1 = a.tp0[k + 1];
  v.bar = a.tbar + (size_t)kTeamBarStride * k;
  return v;
}

// First own column of this block for problem b and the number of own columns
// (columns are dealt cyclically over the team's blocks).
__device__ __forceinline__ void own_range(const TriBatch& a, const TeamView& tv, int b, int& j0,
                                          int& ns) {
  const int G = tv.G, n = a.n[b];
  j0 = ((tv.gb - a.rot[b]) % G + G) % G;
  ns = j0 < n ? (n - 1 - j0) / G + 1 : 0;
}

__device__ __forceinline__ double2* own_col(const TriBatch& a, int b, double2* dsm, int j, int s) {
  const int n = a.n[b];
  return a.soff[b] >= 0 ? dsm + a.soff[b] + (size_t)s * n
                        : a.S0 + (size_t)a.sid[b] * a.slot + (size_t)j * n;
}

// Per-block partials of Re(v_t^H p_t) of problem b, parity t & 1.
__device__ __forceinline__ double* sp_row(const TriBatch& a, int b, int t) {
  return a.sp + (size_t)a.sid[b] * a.sp_stride + (size_t)(t & 1) * gridDim.x;
}

struct HeadShared {
  double red[kHeadGroups][kHeadWarps + 1];
  double2 sc[kHeadGroups][2];
};

// Step t of the team's problems tmem[k0 .. k0 + kHeadGroups - 1] (group q
// serves tmem[k0 + q]), every block of the team alike: column t of the trailing matrix (updated by reflector
// t-1 from the published copy), d_t, and reflector t.  Work vectors: vn = v_t
// (built in place from the column), vo = v_{t-1}, w.  v_{t-1}^H p_{t-1} is the
// sum of the owners' published per-block partials (the same order in every
// block); beta, tau and 1/(alpha - beta) are formed once per problem by the
// group's first thread and passed on in shared memory.  The published p and
// column are loaded in one pass (one L2 round trip per step).
__device__ void tri_heads(const TriBatch& a, const TeamView& tv, int k0, int t, double2* dsm,
                          HeadShared& hs, double2* s_tau, const unsigned char* s_run) {
  const int q = threadIdx.x / kHeadThreads, ht = threadIdx.x % kHeadThreads;
  const int lane = threadIdx.x & 31, hwarp = ht >> 5;
  const bool has = k0 + q < tv.p1;
  const int b = has ? a.tmem[k0 + q] : 0;
  const bool on = has && s_run[b] && t <= a.n[b] - 1;
  const int n = on ? a.n[b] : 0;
  double2* vb = on ? vec_base(a, b, dsm) : dsm;
  double2* vn = vb + (size_t)(t & 1) * n;
  const double2* vo = vb + (size_t)((t + 1) & 1) * n;
  double2* w = vb + 2 * (size_t)n;
  TriPtrs p;
  if (on) p = tri_ptrs(a, b);
  double sg = 0.0;                           // |column|^2 below the subdiagonal
  if (t == 0) {
    if (on) {
      const double2* A = a.A[b];
      for (int i = ht; i < n; i += kHeadThreads) {
        double2 x = A[i];
        x.y = i == 0 ? 0.0 : -x.y;         // column 0 = conj(row 0)
        vn[i] = x;
        if (i >= 2) sg = fma(x.x, x.x, fma(x.y, x.y, sg));
      }
    }
  } else {
    if (on) {
      const double2* Pp = ((t - 1) & 1) ? p.P1 : p.P0;
      const double2* Cp = ((t - 1) & 1) ? p.C1 : p.C0;
      for (int i = t + ht; i < n; i += kHeadThreads) {
        const double2 x = __ldcg(Pp + i);
        w[i] = x;
        vn[i] = __ldcg(Cp + i);            // the column after step t-2's update, for now
        if (i == t) hs.sc[q][0] = x;       // p_{t-1}[t], for w_t in every thread
      }
      if (hwarp == 0) {
        const double* ps = sp_row(a, b, t - 1);
        double S = 0.0;
        for (int g = lane; g < tv.G; g += 32) S += __ldcg(ps + g);
        S = warp_sum(S);
        if (lane == 0) {
          const double2 tau = s_tau[b];
          hs.red[q][kHeadWarps] = 0.5 * (tau.x * tau.x + tau.y * tau.y) * S;
        }
      }
    }
    __syncthreads();
    if (on) {
      // w = tau p - c v_{t-1}; w_t (v_{t-1}[t] = 1) the same bits in every thread;
      // then column t = Cb - v_{t-1} conj(w_t) - w
      const double c = hs.red[q][kHeadWarps];
      const double2 tau = s_tau[b];
      const double2 pt = hs.sc[q][0], vt = vo[t];
      const double2 wt = make_double2(fma(tau.x, pt.x, fma(-tau.y, pt.y, -c * vt.x)),
                                      fma(tau.x, pt.y, fma(tau.y, pt.x, -c * vt.y)));
      for (int i = t + ht; i < n; i += kHeadThreads) {
        const double2 x = w[i], v = vo[i], cb = vn[i];
        const double2 u = make_double2(fma(tau.x, x.x, fma(-tau.y, x.y, -c * v.x)),
                                       fma(tau.x, x.y, fma(tau.y, x.x, -c * v.y)));
        w[i] = u;
        const double2 y = make_double2(fma(-v.x, wt.x, fma(-v.y, wt.y, cb.x - u.x)),
                                       fma(-v.y, wt.x, fma(v.x, wt.y, cb.y - u.y)));
        vn[i] = y;
        if (i >= t + 2) sg = fma(y.x, y.x, fma(y.y, y.y, sg));
      }
    }
  }
  const bool refl = on && t <= n - 2;
  if (refl) {
    sg = warp_sum(sg);
    if (lane == 0) hs.red[q][hwarp] = sg;
  }
  __syncthreads();
  if (refl && ht == 0) {
    double sig = hs.red[q][0];
    for (int k = 1; k < kHeadWarps; ++k) sig += hs.red[q][k];
    const double2 al = vn[t + 1];
    double beta;
    double2 tn, sc;
    if (sig == 0.0 && al.y == 0.0) {
      beta = al.x;                          // already real: H_t = I
      tn = make_double2(0.0, 0.0);
      sc = make_double2(1.0, 0.0);
    } else {
      const double nr = sqrt(al.x * al.x + al.y * al.y + sig);
      beta = al.x >= 0.0 ? -nr : nr;
      const double rb = 1.0 / beta;
      tn = make_double2((beta - al.x) * rb, -al.y * rb);
      const double dx = al.x - beta;        // |Re alpha| + nr: no cancellation
      const double r = 1.0 / fma(dx, dx, al.y * al.y);
      sc = make_double2(dx * r, -al.y * r);  // 1 / (alpha - beta)
    }
    s_tau[b] = tn;
    hs.sc[q][0] = sc;
    hs.sc[q][1] = make_double2(beta, vn[t].x);
    vn[t + 1] = make_double2(1.0, 0.0);
  }
  __syncthreads();
  if (refl) {
    const double2 sc = hs.sc[q][0];
    for (int i = t + 2 + ht; i < n; i += kHeadThreads) {
      const double2 x = vn[i];
      vn[i] = make_double2(fma(x.x, sc.x, -x.y * sc.y), fma(x.x, sc.y, x.y * sc.x));
    }
  }
  __syncthreads();
  if (on && tv.gb == 0) {
    if (refl) {
      if (ht == 0) {
        const double2 bd = hs.sc[q][1];
        p.d[t] = bd.y;
        p.e[t] = bd.x;
        p.e2[t] = bd.x * bd.x;
        p.ddd[t] = dd_of(bd.y);
        p.e2dd[t] = dd_of(bd.x) * dd_of(bd.x);
        p.df[t] = __double2float_rn(bd.y);
        p.e2f[t] = __double2float_rn(bd.x * bd.x);
        p.tau[t] = s_tau[b];
      }
      double2* Vt = p.V + (size_t)t * n;
      for (int i = t + 1 + ht; i < n; i += kHeadThreads) Vt[i] = vn[i];
    } else if (ht == 0) {
      p.d[t] = vn[t].x;                     // t = n - 1
      p.ddd[t] = dd_of(vn[t].x);
      p.df[t] = __double2float_rn(vn[t].x);
    }
  }
}

// Own columns of problem b active at step t (j >= t+1): first slot and count.
__device__ __forceinline__ void active_own(const TriBatch& a, const TeamView& tv, int b, int t,
                                           int& j0, int& smin, int& cb) {
  const int G = tv.G;
  int ns;
  own_range(a, tv, b, j0, ns);
  smin = t + 1 > j0 ? (t + 1 - j0 + G - 1) / G : 0;
  cb = ns > smin ? ns - smin : 0;
}

// Own columns j >= t+1, one warp per column: update by reflector t-1 (rows
// > t), p_j = col_j^H v_t, publication of p_j and of column t+1, and the
// block's partial of Re(v_t^H p_t) per problem (over its own columns, in
// column order), for the team's problems.
__device__ void tri_body(const TriBatch& a, const TeamView& tv, int t, double2* dsm,
                         double* contrib, const unsigned char* s_run) {
  const int G = tv.G, lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int C = 0;
  for (int k = tv.p0; k < tv.p1; ++k) {
    const int b = a.tmem[k];
    if (!s_run[b] || t > a.n[b] - 2) continue;
    int j0, smin, cb;
    active_own(a, tv, b, t, j0, smin, cb);
    C += cb;
  }
  for (int ci = wid; ci < C; ci += kTriWarps) {
    // column ci -> problem b, column j, slot s
    int b = 0, j = 0, s = 0, rest = ci;
    for (int k = tv.p0; k < tv.p1; ++k) {
      b = a.tmem[k];
      if (!s_run[b] || t > a.n[b] - 2) continue;
      int j0, smin, cb;
      active_own(a, tv, b, t, j0, smin, cb);
      if (rest < cb) {
        s = smin + rest;
        j = j0 + s * G;
        break;
      }
      rest -= cb;
    }
    const int n = a.n[b];
    double2* col = own_col(a, b, dsm, j, s);
    const double2* vb = vec_base(a, b, dsm);
    const double2* vn = vb + (size_t)(t & 1) * n;
    const double2* vo = vb + (size_t)((t + 1) & 1) * n;
    const double2* w = vb + 2 * (size_t)n;
    const TriPtrs p = tri_ptrs(a, b);
    double2* Cb = (t & 1) ? p.C1 : p.C0;
    const bool upd = t >= 1, pub = (j == t + 1);
    const double2 wj = upd ? conjx(w[j]) : make_double2(0.0, 0.0);
    const double2 vj = upd ? conjx(vo[j]) : make_double2(0.0, 0.0);
    double ax = 0.0, ay = 0.0;
    for (int i = t + 1 + lane; i < n; i += 32) {
      double2 x = col[i];
      if (upd) {                            // x -= vo_i conj(w_j) + w_i conj(vo_j)
        const double2 v = vo[i], u = w[i];
        x.x = fma(-v.x, wj.x, fma(v.y, wj.y, fma(-u.x, vj.x, fma(u.y, vj.y, x.x))));
        x.y = fma(-v.x, wj.y, fma(-v.y, wj.x, fma(-u.x, vj.y, fma(-u.y, vj.x, x.y))));
        col[i] = x;
      }
      const double2 v = vn[i];
      ax = fma(x.x, v.x, fma(x.y, v.y, ax));      // conj(x) v
      ay = fma(x.x, v.y, fma(-x.y, v.x, ay));
      if (pub) Cb[i] = x;
    }
    ax = warp_sum(ax);
    ay = warp_sum(ay);
    if (lane == 0) {
      ((t & 1) ? p.P1 : p.P0)[j] = make_double2(ax, ay);
      const double2 vnj = vn[j];
      contrib[ci] = fma(vnj.x, ax, vnj.y * ay);   // Re(conj(v_t[j]) p_j)
    }
  }
  __syncthreads();
  // per-problem partials, one thread per problem, own columns in order
  for (int k = tv.p0 + (int)threadIdx.x; k < tv.p1; k += blockDim.x) {
    const int b = a.tmem[k];
    if (!s_run[b] || t > a.n[b] - 2) continue;
    int first = 0;
    for (int kq = tv.p0; kq < k; ++kq) {
      const int q = a.tmem[kq];
      if (!s_run[q] || t > a.n[q] - 2) continue;
      int j0, smin, cb;
      active_own(a, tv, q, t, j0, smin, cb);
      first += cb;
    }
    int j0, smin, cb;
    active_own(a, tv, b, t, j0, smin, cb);
    double acc = 0.0;
    for (int i = 0; i < cb; ++i) acc += contrib[first + i];
    sp_row(a, b, t)[tv.gb] = acc;
  }
}

__global__ void __launch_bounds__(kTriThreads, 1) k_hh_tridiag(TriBatch a) {
  extern __shared__ double2 dsm[];
  __shared__ HeadShared hs;
  __shared__ double2 s_tau[kMaxBatch];
  __shared__ unsigned char s_run[kMaxBatch];
  const int tid = threadIdx.x, nt = blockDim.x;
  double* contrib = reinterpret_cast<double*>(dsm + a.coff);
  const TeamView tv = team_view(a);
  unsigned epoch = 0;
  int nrun = 0;
  for (int k = tv.p0; k < tv.p1; ++k) {
    const int b = a.tmem[k];
    const bool r = tri_run(a, b);
    if (tid == 0) {
      s_run[b] = r;
      s_tau[b] = make_double2(0.0, 0.0);
    }
    if (r && a.n[b] > nrun) nrun = a.n[b];
  }
  __syncthreads();
  // own columns: column j = conj(row j) of the Hermitian input
  for (int k = tv.p0; k < tv.p1; ++k) {
    const int b = a.tmem[k];
    if (!s_run[b]) continue;
    int j0, ns;
    own_range(a, tv, b, j0, ns);
    const int n = a.n[b];
    const double2* A = a.A[b];
    for (int s = 0; s < ns; ++s) {
      const int j = j0 + s * tv.G;
      double2* col = own_col(a, b, dsm, j, s);
      for (int i = tid; i < n; i += nt) {
        double2 x = A[(size_t)j * n + i];
        x.y = i == j ? 0.0 : -x.y;
        col[i] = x;
      }
    }
  }
  __syncthreads();
  for (int t = 0; t < nrun; ++t) {
    for (int k0 = tv.p0; k0 < tv.p1; k0 += kHeadGroups)
      tri_heads(a, tv, k0, t, dsm, hs, s_tau, s_run);
    tri_body(a, tv, t, dsm, contrib, s_run);
    if (t + 1 < nrun) {
      if (tv.G == 1) {
        __syncthreads();
      } else if (!blocks_barrier(tv.bar, epoch, (unsigned)tv.G, a.status, a.spins)) {
        return;
      }
    }
  }
  if (tv.gb == 0 && tid == 0) {
    long long k = 0;
    for (int q = tv.p0; q < tv.p1; ++q) k += s_run[a.tmem[q]];
    atomicAdd(reinterpret_cast<unsigned long long*>(a.stats + 6), (unsigned long long)k);
  }
}

// ---- stage 2: eigenvalues of T -------------------------------------------------
// Number of eigenvalues of T below x: the number of negative pivots of the
// LDL^T factorisation of T - x I, q_0 = d_0 - x, q_k = (d_k - x) -
// e_{k-1}^2 / q_{k-1} (Sylvester's law of inertia); a pivot of modulus below
// pivmin is replaced by -pivmin.  The computed count is exact for T with
// every d_k - x and e_k^2 perturbed by a few units of the arithmetic's last
// place (Kahan; LAPACK's dstebz), so x is located to within that perturbation
// of ||T||.  On this chip a dependent FP64 operation takes ~67 cycles and an
// FP64 division ~670 (measured), FP32 ones ~5, so the count runs in FP32 to
// about 2^-16 ||T|| and then in double-float arithmetic (about 2^-46 per
// operation) to 2^-43 ||T||, no FP64 operation in the loops.
constexpr float kPivMin32 = 0x1p-100f;
constexpr double kBisF32Rel = 0x1p-16;   // FP32 rounds down to this width / ||T||
constexpr double kBisF32Pad = 0x1p-17;   // then widened by this much / ||T|| on each side
constexpr double kBisDDRel = 0x1p-43;    // double-float rounds down to this width / ||T||

__device__ __forceinline__ int sturm_count32(const float* __restrict__ d,
                                             const float* __restrict__ e2, int n, float x) {
  float q = __ldg(d) - x;
  int cnt = 0;
  for (int i = 1;; ++i) {
    if (fabsf(q) < kPivMin32) q = -kPivMin32;
    cnt += q < 0.0f;
    if (i >= n) break;
    q = (__ldg(d + i) - x) - __fdividef(__ldg(e2 + i - 1), q);
  }
  return cnt;
}
__device__ __forceinline__ int sturm_count_dd(const dd* __restrict__ d, const dd* __restrict__ e2,
                                              int n, dd x) {
  dd q = d[0] - x;
  int cnt = 0;
  for (int i = 1;; ++i) {
    if (fabsf(q.hi) < kPivMin32) q = dd(-kPivMin32, 0.0f);
    cnt += q.hi < 0.0f;
    if (i >= n) break;
    q = (d[i] - x) - ddiv(e2[i - 1], q);
  }
  return cnt;
}

// One warp per eigenvalue (every eigenvalue its own warp: one wave).  The
// lanes count at L points per round, so a round narrows the bracket L + 1
// times; the bracket invariant is count(lo) <= j < count(hi).
__global__ void __launch_bounds__(32) k_tri_bisect(TriBatch a) {
  constexpr int L = kBisLanes;
  static_assert(L == 32, "one warp per eigenvalue");
  const int l = threadIdx.x;
  const unsigned mask = 0xffffffffu;
  const int item = blockIdx.x;
  if (item >= a.off[a.np]) return;
  const int b = find_prob(a.off, a.np, item);
  if (!tri_run(a, b)) return;
  const int n = a.n[b], j = item - a.off[b];
  const TriPtrs p = tri_ptrs(a, b);
  // Gershgorin interval
  double glo = INFINITY, ghi = -INFINITY;
  for (int i = l; i < n; i += L) {
    const double r = (i > 0 ? fabs(p.e[i - 1]) : 0.0) + (i < n - 1 ? fabs(p.e[i]) : 0.0);
    glo = fmin(glo, p.d[i] - r);
    ghi = fmax(ghi, p.d[i] + r);
  }
#pragma unroll
  for (int o = 1; o < L; o <<= 1) {
    glo = fmin(glo, __shfl_xor_sync(mask, glo, o));
    ghi = fmax(ghi, __shfl_xor_sync(mask, ghi, o));
  }
  const double nrm = fmax(fmax(fabs(glo), fabs(ghi)), 1e-290);
  const double pad = 2.0 * kEps * nrm + 1e-290;
  glo -= pad;
  ghi += pad;
  // a round: counts at L interior points (or, with ends, at L points from lo
  // to hi inclusive); returns false when the ends do not bracket j
  auto narrow = [&](double& lo, double& hi, int cnt, double x) {
    double nlo = lo, nhi = hi;
    bool above = false;
#pragma unroll 4
    for (int k = 0; k < L; ++k) {
      const double xk = __shfl_sync(mask, x, k);
      const int ck = __shfl_sync(mask, cnt, k);
      if (!above) {
        if (ck <= j) nlo = xk;
        else { nhi = xk; above = true; }
      }
    }
    lo = nlo;
    hi = nhi;
  };
  // FP32 rounds
  double lo = glo, hi = ghi;
  {
    float lo32 = __double2float_rd(lo), hi32 = __double2float_ru(hi);
    const float w32 = (float)(kBisF32Rel * nrm);
    for (int round = 0; round < 12 && hi32 - lo32 > w32; ++round) {
      const float x = lo32 + (hi32 - lo32) * ((float)(l + 1) / (float)(L + 1));
      const int cnt = sturm_count32(p.df, p.e2f, n, x);
      double dlo = lo32, dhi = hi32;
      narrow(dlo, dhi, cnt, (double)x);
      lo32 = (float)dlo;
      hi32 = (float)dhi;
    }
    lo = fmax((double)lo32 - kBisF32Pad * nrm, glo);
    hi = fmin((double)hi32 + kBisF32Pad * nrm, ghi);
  }
  // double-float rounds; the first one includes both ends as a check
  {
    const double x = lo + (hi - lo) * ((double)l / (double)(L - 1));
    const int cnt = sturm_count_dd(p.ddd, p.e2dd, n, dd_of(x));
    const int c0 = __shfl_sync(mask, cnt, 0), cL = __shfl_sync(mask, cnt, L - 1);
    if (c0 <= j && cL > j) {
      narrow(lo, hi, cnt, x);
    } else {
      lo = glo;                              // the FP32 bracket missed: start over
      hi = ghi;
    }
  }
  const double tol = kBisDDRel * nrm;
  for (int round = 0; round < kBisMaxRounds && hi - lo > tol; ++round) {
    const double x = lo + (hi - lo) * ((double)(l + 1) / (double)(L + 1));
    const int cnt = sturm_count_dd(p.ddd, p.e2dd, n, dd_of(x));
    narrow(lo, hi, cnt, x);
  }
  if (l == 0) {
    const double lam = 0.5 * (lo + hi);
    p.lam[j] = lam;
    a.w[b][j] = lam;
  }
}

// ---- stage 3: eigenvectors of T ---------------------------------------------------
// Uniform in [-1, 1) from (k, i): the splitmix64 finaliser of a Weyl sequence.
__device__ __forceinline__ double start_entry(unsigned long long k, unsigned long long i) {
  unsigned long long x = k * 0x9E3779B97F4A7C15ull + (i + 1) * 0xD1B54A32D192ED03ull;
  x ^= x >> 30; x *= 0xBF58476D1CE4E5B9ull;
  x ^= x >> 27; x *= 0x94D049BB133111EBull;
  x ^= x >> 31;
  return (double)(x >> 11) * (1.0 / 4503599627370496.0) - 1.0;
}

// LU factors with partial pivoting of T - lam I for column k (row stride n):
// U0 = 1 / (pivot), U1 = first superdiagonal of U, U2 = the multiplier of
// the row operation, its lowest mantissa bit set when rows i and i+1 were
// swapped (then U's second superdiagonal is e_{i+1}, else 0).  One
// reciprocal per row; a zero pivot is replaced by pert.
__device__ __forceinline__ double pack_piv(double l, bool piv) {
  return __longlong_as_double((__double_as_longlong(l) & ~1ll) | (long long)piv);
}
__device__ __forceinline__ bool piv_of(double l) { return (__double_as_longlong(l) & 1ll) != 0; }

__device__ __forceinline__ void tri_factor(const TriPtrs& p, int n, int k, double lam, double pert) {
  const size_t sn = (size_t)n;
  double cur0 = p.d[0] - lam, cur1 = n > 1 ? p.e[0] : 0.0;
  for (int i = 0; i < n - 1; ++i) {
    const double sub = p.e[i], nd = p.d[i + 1] - lam;
    const double nsup = i + 1 < n - 1 ? p.e[i + 1] : 0.0;
    const bool piv = fabs(sub) > fabs(cur0);
    const double c0 = cur0 == 0.0 ? pert : cur0;
    const double r = 1.0 / (piv ? sub : c0);
    const double l = (piv ? cur0 : sub) * r;
    const size_t e = (size_t)i * sn + k;
    p.U0[e] = r;
    p.U1[e] = piv ? nd : cur1;
    p.U2[e] = pack_piv(l, piv);
    const double n0 = piv ? fma(-l, nd, cur1) : fma(-l, cur1, nd);
    cur1 = piv ? -l * nsup : nsup;
    cur0 = n0;
  }
  p.U0[(size_t)(n - 1) * sn + k] = 1.0 / (cur0 == 0.0 ? pert : cur0);
}

// y <- (T - lam I)^{-1} y on column k of Y with the stored factors.
__device__ __forceinline__ void tri_solve(const TriPtrs& p, int n, int k) {
  double* Y = p.Y;
  const size_t sn = (size_t)n;
  double rc = Y[k];
  for (int i = 0; i < n - 1; ++i) {
    const size_t e = (size_t)i * sn + k;
    const double lv = p.U2[e], rn = Y[e + sn];
    if (piv_of(lv)) {
      Y[e] = rn;
      rc = fma(-lv, rn, rc);
    } else {
      Y[e] = rc;
      rc = fma(-lv, rc, rn);
    }
  }
  Y[(size_t)(n - 1) * sn + k] = rc;
  double y1 = 0.0, y2 = 0.0;                // y[i+1], y[i+2]
  for (int i = n - 1; i >= 0; --i) {
    const size_t e = (size_t)i * sn + k;
    // the last row has no superdiagonal (its U1 and U2 entries are never formed)
    const double u1 = i + 1 < n ? p.U1[e] : 0.0;
    const double u2 = (i + 2 < n && piv_of(p.U2[e])) ? p.e[i + 1] : 0.0;
    const double yi = (Y[e] - u1 * y1 - u2 * y2) * p.U0[e];
    Y[e] = yi;
    y2 = y1;
    y1 = yi;
  }
}

// One thread per eigenvalue; the first of a cluster does the whole cluster.
// Blocks of kVecThreads spread the serial work over the SMs.
__global__ void __launch_bounds__(kVecThreads, 1) k_tri_vectors(TriBatch a) {
  const int item = blockIdx.x * kVecThreads + threadIdx.x;
  if (item >= a.off[a.np]) return;
  const int b = find_prob(a.off, a.np, item);
  if (!tri_run(a, b)) return;
  const int n = a.n[b], j = item - a.off[b];
  const TriPtrs p = tri_ptrs(a, b);
  const double* lam = p.lam;
  const double nrm = fmax(fmax(fabs(lam[0]), fabs(lam[n - 1])), 1e-300);
  const double tight = kTightRel * nrm;
  if (j > 0 && lam[j] - lam[j - 1] <= tight) return;   // not the first of its cluster
  int end = j + 1;
  while (end < n && lam[end] - lam[end - 1] <= tight) ++end;
  const double pert = kEps * nrm;
  const size_t sn = (size_t)n;
  double* Y = p.Y;
  for (int k = j; k < end; ++k) {
    for (int i = 0; i < n; ++i) Y[(size_t)i * sn + k] = start_entry((unsigned long long)k, i);
    tri_factor(p, n, k, lam[k], pert);
    for (int it = 0; it < kInvIters; ++it) {
      tri_solve(p, n, k);
      for (int c = j; c < k; ++c) {          // against the cluster's earlier vectors
        double dot = 0.0;
        for (int i = 0; i < n; ++i) dot = fma(Y[(size_t)i * sn + c], Y[(size_t)i * sn + k], dot);
        for (int i = 0; i < n; ++i) Y[(size_t)i * sn + k] = fma(-dot, Y[(size_t)i * sn + c], Y[(size_t)i * sn + k]);
      }
      double s = 0.0;
      if (it + 1 < kInvIters) {
        for (int i = 0; i < n; ++i) s = fmax(s, fabs(Y[(size_t)i * sn + k]));
      } else {
        for (int i = 0; i < n; ++i) s = fma(Y[(size_t)i * sn + k], Y[(size_t)i * sn + k], s);
        s = sqrt(s);
      }
      if (!(s > 0.0) || !isfinite(s)) {
        flag_status(a.status, SKY_ENOCONV);
        s = 1.0;
      }
      const double r = 1.0 / s;
      for (int i = 0; i < n; ++i) Y[(size_t)i * sn + k] *= r;
    }
  }
}

// One first-order Loewdin step on the columns of Y within each eigenvalue's
// window: Yout[:, j] = Yin[:, j] (3 - G_jj)/2 - sum_{k != j} G_kj Yin[:, k] / 2.
__global__ void __launch_bounds__(kWinThreads) k_tri_window(TriBatch a, int pass) {
  __shared__ double gpart[kWinThreads / 32][2 * kWinMax + 1];
  __shared__ double coef[2 * kWinMax + 1];
  const int item = blockIdx.x;
  const int b = find_prob(a.off, a.np, item);
  if (!tri_run(a, b)) return;
  const int n = a.n[b], j = item - a.off[b];
  const TriPtrs p = tri_ptrs(a, b);
  const double* Yin = pass ? p.Y2 : p.Y;
  double* Yout = pass ? p.Y : p.Y2;
  const double* lam = p.lam;
  const double gw = kWinRel * fmax(fabs(lam[0]), fabs(lam[n - 1]));
  int lo = j, hi = j;
  while (lo > 0 && j - lo < kWinMax && lam[j] - lam[lo - 1] <= gw) --lo;
  while (hi < n - 1 && hi - j < kWinMax && lam[hi + 1] - lam[j] <= gw) ++hi;
  const int K = hi - lo + 1;
  const int lane = threadIdx.x & 31, wq = threadIdx.x >> 5;
  const size_t sn = (size_t)n;
  double acc[kWinChunks];
#pragma unroll
  for (int c = 0; c < kWinChunks; ++c) acc[c] = 0.0;
  for (int i = wq; i < n; i += kWinThreads / 32) {
    const double* row = Yin + (size_t)i * sn;
    const double yj = row[j];
#pragma unroll
    for (int c = 0; c < kWinChunks; ++c) {
      const int t = lane + 32 * c;
      if (t < K) acc[c] = fma(row[lo + t], yj, acc[c]);
    }
  }
#pragma unroll
  for (int c = 0; c < kWinChunks; ++c) {
    const int t = lane + 32 * c;
    if (t < K) gpart[wq][t] = acc[c];
  }
  __syncthreads();
  for (int t = threadIdx.x; t < K; t += kWinThreads) {
    double g = gpart[0][t];
    for (int q = 1; q < kWinThreads / 32; ++q) g += gpart[q][t];
    coef[t] = (lo + t == j) ? 1.5 - 0.5 * g : -0.5 * g;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += kWinThreads) {
    const double* row = Yin + (size_t)i * sn + lo;
    double s = 0.0;
    for (int t = 0; t < K; ++t) s = fma(coef[t], row[t], s);
    Yout[(size_t)i * sn + j] = s;
  }
}

// ---- back-transformation: Z = H_0 H_1 ... H_{n-2} Y, one warp per column ----------
__global__ void __launch_bounds__(kBackWarps * 32) k_hh_back(TriBatch a, int zstride) {
  extern __shared__ double2 dsm[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  double2* z = dsm + (size_t)wid * zstride;
  const int nw = gridDim.x * (blockDim.x >> 5);
  const int total = a.off[a.np];
  for (int it = wid * gridDim.x + blockIdx.x; it < total; it += nw) {
    const int b = find_prob(a.off, a.np, it);
    if (!tri_run(a, b)) continue;
    const int n = a.n[b], col = it - a.off[b];
    const TriPtrs p = tri_ptrs(a, b);
    for (int i = lane; i < n; i += 32) z[i] = make_double2(p.Y[(size_t)i * n + col], 0.0);
    for (int k = n - 2; k >= 0; --k) {
      const double2 tau = p.tau[k];
      if (tau.x == 0.0 && tau.y == 0.0) continue;
      const double2* v = p.V + (size_t)k * n;
      const int i0 = ((k + 1) >> 5) * 32 + lane;
      double sx = 0.0, sy = 0.0;
      for (int i = i0; i < n; i += 32) {
        if (i <= k) continue;
        const double2 vi = v[i], zi = z[i];
        sx = fma(vi.x, zi.x, fma(vi.y, zi.y, sx));     // conj(v) z
        sy = fma(vi.x, zi.y, fma(-vi.y, zi.x, sy));
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        sx += __shfl_xor_sync(0xffffffffu, sx, o);
        sy += __shfl_xor_sync(0xffffffffu, sy, o);
      }
      const double2 f = cmul(tau, make_double2(sx, sy));
      for (int i = i0; i < n; i += 32) {
        if (i <= k) continue;
        const double2 vi = v[i];
        double2 zi = z[i];
        zi.x = fma(-vi.x, f.x, fma(vi.y, f.y, zi.x));     // z -= v f
        zi.y = fma(-vi.x, f.y, fma(-vi.y, f.x, zi.y));
        z[i] = zi;
      }
    }
    double2* Z = a.Z[b];
    for (int i = lane; i < n; i += 32) Z[(size_t)i * n + col] = z[i];
    __syncwarp();
  }
}

__global__ void k_tri_reset(unsigned* bar) { bar[(size_t)kTeamBarStride * threadIdx.x] = 0u; }

// A problem of n states keeps its work vectors in global memory when they
// alone (with the per-column partials) exceed the shared-memory budget.
bool tri_vectors_global(int n) {
  return (3 * (size_t)n + (n + 1) / 2 + 1) * sizeof(double2) > kTriSmemMax;
}

// double2 elements of the global work vectors for the problems of a batch
// of nb problems of up to m states on nsm blocks: needed when one problem,
// or the tridiagonal route's largest batch (8 problems) of them, does not fit
// in shared memory (0 otherwise).
size_t tri_vec_elems(int m, int nb, int nsm) {
  const int k = nb < 8 ? nb : 8;
  const size_t one = (3 * (size_t)m + (m + 1) / 2 + 1) * sizeof(double2);
  return (tri_vectors_global(m) || k * one > kTriSmemMax) ? (size_t)k * nsm * 3 * (size_t)m : 0;
}

// Shared-memory opt-in of the two kernels that take more than 48 KB (once per
// context, outside any stream capture).
sky_status tri_init(Ctx* c) {
  cudaError_t e = cudaFuncSetAttribute(k_hh_tridiag, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)kTriSmemMax);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_hh_back, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTriSmemMax);
  return cuda_check(c, e, "tridiagonal solver attributes");
}

// ---- teams of blocks for batches of many problems ----------------------------------
// With one team, every block takes part in every problem's steps and the
// slowest problem sets the pace of all: n_max steps, each with the head work
// of every problem.  A batch of more than kTeamMin problems (the many boxes of
// twist-averaged runs) is split instead: a problem whose work needs several
// blocks gets a team of its own, smaller ones share one-block teams (no
// barrier at all), each team stepping at its own pace.  The split minimises
// the largest estimated team time
//   steps x (per-step latency) + sum over its problems of 4 n^3 FMAs / rate,
// by bisection on the time target: problems are taken largest first, teams
// of several blocks sized to the target, the rest packed first-fit into
// one-block teams whose work vectors fit in shared memory.
constexpr int kTeamMin = 8;
constexpr double kTeamFma = 3.4e9;      // FP64 FMAs per second of one block (one per SM)
constexpr double kTeamStep1 = 1.5e-6;   // seconds per step of a one-block team
constexpr double kTeamStepG = 5.0e-6;   // seconds per step of a team with a barrier
constexpr double kTeamHead = 1.0e-6;    // per step and further group of kHeadGroups problems
constexpr int kTeamMinCols = 4;         // own columns per block of a team at least

struct TeamPlan {
  int nteam;
  int mem[kMaxBatch];
  int p0[kMaxBatch + 1];
  int g0[kMaxBatch + 1];
};

static double team_work(int n) { return 4.0 * (double)n * n * n / kTeamFma; }
static size_t team_vec(int n) { return 3 * (size_t)n + (size_t)(n + 1) / 2 + 1; }   // double2

// Estimated time of a team of g blocks for problems mem[k0 .. k1).
static double team_time(const int* n, const int* mem, int k0, int k1, int g) {
  int nmax = 0;
  double w = 0.0;
  for (int k = k0; k < k1; ++k) {
    nmax = n[mem[k]] > nmax ? n[mem[k]] : nmax;
    w += team_work(n[mem[k]]);
  }
  const int groups = (k1 - k0 + kHeadGroups - 1) / kHeadGroups;
  const double step = (g > 1 ? kTeamStepG : kTeamStep1) + kTeamHead * (groups - 1);
  return nmax * step + w / g;
}

// Teams for the target time T (problems in `order`, largest first); returns
// the blocks used, or a number above `blocks` when T cannot be met.
static int plan_at(int np, const int* n, const int* order, double T, size_t budget, TeamPlan& p) {
  int used = 0, k = 0;
  p.nteam = 0;
  bool packed[kMaxBatch];
  for (int i = 0; i < np; ++i) {
    const int b = order[i];
    packed[b] = team_work(n[b]) + n[b] * kTeamStep1 <= T;
    if (packed[b]) continue;
    const double room = T - n[b] * kTeamStepG;
    const int gmax = n[b] / kTeamMinCols > 2 ? n[b] / kTeamMinCols : 2;
    if (room <= 0.0) return 1 << 30;
    const double gf = team_work(n[b]) / room;
    if (gf > gmax) return 1 << 30;
    int g = (int)std::ceil(gf);
    g = g < 2 ? 2 : g;
    p.p0[p.nteam] = k;
    p.g0[p.nteam] = used;
    p.mem[k++] = b;
    used += g;
    ++p.nteam;
  }
  // first fit, largest first, into one-block teams
  int bin_of[kMaxBatch], nbin = 0;
  double bw[kMaxBatch];
  int bn[kMaxBatch], bk[kMaxBatch];
  size_t bv[kMaxBatch];
  for (int i = 0; i < np; ++i) {
    const int b = order[i];
    if (!packed[b]) continue;
    int f = -1;
    for (int q = 0; q < nbin && f < 0; ++q) {
      const int groups = (bk[q] + 1 + kHeadGroups - 1) / kHeadGroups;
      const double t = bn[q] * (kTeamStep1 + kTeamHead * (groups - 1)) + bw[q] + team_work(n[b]);
      if (t <= T && bv[q] + team_vec(n[b]) <= budget) f = q;
    }
    if (f < 0) {
      if (team_vec(n[b]) > budget) return 1 << 30;
      f = nbin++;
      bw[f] = 0.0; bn[f] = n[b]; bk[f] = 0; bv[f] = 0;
    }
    bw[f] += team_work(n[b]);
    bk[f] += 1;
    bv[f] += team_vec(n[b]);
    bin_of[b] = f;
  }
  for (int q = 0; q < nbin; ++q) {
    p.p0[p.nteam] = k;
    p.g0[p.nteam] = used++;
    for (int i = 0; i < np; ++i)
      if (packed[order[i]] && bin_of[order[i]] == q) p.mem[k++] = order[i];
    ++p.nteam;
  }
  p.p0[p.nteam] = k;
  p.g0[p.nteam] = used;
  return used;
}

// The team split of np problems over `blocks` blocks (false if none fits).
static bool plan_teams(int np, const int* n, int blocks, size_t budget, TeamPlan& p) {
  int order[kMaxBatch];
  for (int b = 0; b < np; ++b) order[b] = b;
  std::sort(order, order + np, [&](int x, int y) { return n[x] != n[y] ? n[x] > n[y] : x < y; });
  // an upper time bound that fits (1 s covers the usual batches on a full GPU;
  // larger batches on fewer blocks need longer), then bisection
  double hi = 1.0, lo = 0.0;
  while (plan_at(np, n, order, hi, budget, p) > blocks) {
    lo = hi;
    hi *= 2.0;
    if (hi > 1e7) return false;   // no split fits (shared memory bounds the packing)
  }
  for (int it = 0; it < 48; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (plan_at(np, n, order, mid, budget, p) <= blocks) hi = mid; else lo = mid;
  }
  int used = plan_at(np, n, order, hi, budget, p);
  // spare blocks to the slowest single-problem teams
  while (used < blocks) {
    int best = -1;
    double bt = 0.0;
    for (int t = 0; t < p.nteam; ++t) {
      const int g = p.g0[t + 1] - p.g0[t];
      if (p.p0[t + 1] - p.p0[t] != 1 || g + 1 > n[p.mem[p.p0[t]]] / kTeamMinCols) continue;
      const double tt = team_time(n, p.mem, p.p0[t], p.p0[t + 1], g);
      if (tt > bt) { bt = tt; best = t; }
    }
    if (best < 0) break;
    for (int t = best + 1; t <= p.nteam; ++t) p.g0[t] += 1;
    ++used;
  }
  return true;
}

// The team split of a batch on `blocks` blocks for callers (sky_tri_team_plan):
// the number of teams, 0 if it cannot be split.
int tri_team_plan(int np, const int* n, int blocks, int* team, int* first, int* count) {
  if (np < 1 || np > kMaxBatch || blocks < 1 || !n || !team || !first || !count) return 0;
  for (int b = 0; b < np; ++b)
    if (n[b] < 1 || tri_vectors_global(n[b])) return 0;
  TeamPlan tp;
  if (!plan_teams(np, n, blocks, kTriSmemMax / sizeof(double2) - 64, tp)) return 0;
  for (int t = 0; t < tp.nteam; ++t) {
    first[t] = tp.g0[t];
    count[t] = tp.g0[t + 1] - tp.g0[t];
    for (int k = tp.p0[t]; k < tp.p0[t + 1]; ++k) team[tp.mem[k]] = t;
  }
  return tp.nteam;
}

// One launch sequence for the problems idx[0..np) of a batch (their vectors fit).
static sky_status tri_group(Ctx* c, int np, const int* idx, const double2* const* A, const int* n,
                            double* const* w, double2* const* Z, const int* run, int run_stride,
                            const bool* gvec) {
  TriBatch a;
  a.np = np;
  a.off[0] = 0;
  long long ntot = 0;
  int nmax = 1;
  for (int q = 0; q < np; ++q) {
    const int b = idx[q];
    a.A[q] = A[b]; a.w[q] = w[b]; a.Z[q] = Z[b]; a.n[q] = n[b]; a.sid[q] = b;
    a.off[q + 1] = a.off[q] + n[b];
    ntot += n[b];
    if (n[b] > nmax) nmax = n[b];
  }
  if (ntot == 0) return SKY_OK;
  int G = (int)(ntot < c->num_sms ? ntot : c->num_sms);
  size_t used = 0;
  a.gvec = c->d_trivec;
  a.gvec_stride = 3 * (size_t)c->tri_m;
  if (np > kTeamMin) {
    // teams: the per-column partials first (one region for every team), then
    // each team's work vectors and own columns while they fit
    TeamPlan tp;
    const size_t budget = kTriSmemMax / sizeof(double2);
    G = c->num_sms;
    if (!plan_teams(np, a.n, G, budget - 64, tp)) return SKY_EUNSUPPORTED;
    G = tp.g0[tp.nteam];
    a.nteam = tp.nteam;
    size_t cmax = 0;
    for (int t = 0; t <= tp.nteam; ++t) {
      a.tp0[t] = tp.p0[t];
      a.tg0[t] = tp.g0[t];
    }
    for (int k = 0; k < np; ++k) a.tmem[k] = tp.mem[k];
    for (int t = 0; t < tp.nteam; ++t) {
      const int g = tp.g0[t + 1] - tp.g0[t];
      size_t own = 0;
      for (int k = tp.p0[t]; k < tp.p0[t + 1]; ++k) own += (a.n[tp.mem[k]] + g - 1) / g;
      cmax = own > cmax ? own : cmax;
    }
    a.coff = 0;
    const size_t base = (cmax + 1) / 2 + 1;
    used = base;
    for (int t = 0; t < tp.nteam; ++t) {
      const int g = tp.g0[t + 1] - tp.g0[t];
      size_t u = base;
      for (int k = tp.p0[t]; k < tp.p0[t + 1]; ++k) {
        const int q = tp.mem[k];
        if (gvec[idx[q]]) return SKY_EUNSUPPORTED;
        a.voff[q] = (int)u;
        u += 3 * (size_t)a.n[q];
        a.rot[q] = 0;
      }
      if (u > budget) return SKY_EUNSUPPORTED;
      for (int k = tp.p0[t]; k < tp.p0[t + 1]; ++k) {
        const int q = tp.mem[k];
        const size_t need = (size_t)((a.n[q] + g - 1) / g) * a.n[q];
        if (u + need <= budget) {
          a.soff[q] = (int)u;
          u += need;
        } else {
          a.soff[q] = -1;
        }
      }
      used = u > used ? u : used;
    }
    a.tbar = c->d_tbar;
  } else {
    // one team of all blocks.  Shared memory: three work vectors per problem
    // (in global memory for a problem whose vectors alone exceed it), then own
    // columns while they fit
    int maxown = 0;
    for (int q = 0; q < np; ++q) {
      if (gvec[idx[q]]) {
        a.voff[q] = -1;
      } else {
        a.voff[q] = (int)used;
        used += 3 * (size_t)a.n[q];
      }
      maxown += (a.n[q] + G - 1) / G;
    }
    a.coff = (int)used;
    used += (size_t)(maxown + 1) / 2;
    int rot = 0;
    for (int q = 0; q < np; ++q) {
      const size_t need = (size_t)((a.n[q] + G - 1) / G) * a.n[q];
      if ((used + need) * sizeof(double2) <= kTriSmemMax) {
        a.soff[q] = (int)used;
        used += need;
      } else {
        a.soff[q] = -1;
      }
      a.rot[q] = rot;
      rot = (rot + a.n[q]) % G;
    }
    a.nteam = 1;
    a.tp0[0] = 0; a.tp0[1] = np;
    a.tg0[0] = 0; a.tg0[1] = G;
    for (int q = 0; q < np; ++q) a.tmem[q] = q;
    a.tbar = c->d_bar;
  }
  const int zstride = nmax + (nmax & 1);
  int back_warps = kBackWarps;
  while (back_warps > 1 && (size_t)back_warps * zstride * sizeof(double2) > kTriSmemMax) back_warps >>= 1;
  a.S0 = c->d_eigA[0]; a.S1 = c->d_eigA[1]; a.S2 = c->d_eigV; a.slot = c->eig_slot;
  a.T = c->d_trid; a.tslot = c->tri_slot; a.m = c->tri_m;
  a.sp = c->d_eigpart; a.sp_stride = (size_t)2 * c->eig_grid_max;
  a.run = run; a.run_stride = run_stride;
  a.bar = c->d_bar; a.status = c->d_status; a.spins = c->wait_spins; a.stats = c->d_stats;
  // run flags are indexed by the batch position of each problem
  if (run) {
    bool ident = true;
    for (int q = 0; q < np; ++q) ident = ident && idx[q] == q;
    if (!ident) return SKY_EUNSUPPORTED;
  }
  cudaError_t e;
  k_tri_reset<<<1, a.nteam, 0, c->stream>>>(a.tbar);
  note_launch();
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_check(c, e, "tridiagonal reset");
  void* args[] = {&a};
  note_launch();
  e = cudaLaunchCooperativeKernel((const void*)k_hh_tridiag, dim3(G), dim3(kTriThreads), args,
                                  used * sizeof(double2), c->stream);
  if (e != cudaSuccess) return cuda_check(c, e, "householder tridiagonalisation");
  k_tri_bisect<<<(unsigned)ntot, 32, 0, c->stream>>>(a);
  k_tri_vectors<<<div_up(ntot, kVecThreads), kVecThreads, 0, c->stream>>>(a);
  k_tri_window<<<(unsigned)ntot, kWinThreads, 0, c->stream>>>(a, 0);
  k_tri_window<<<(unsigned)ntot, kWinThreads, 0, c->stream>>>(a, 1);
  // columns spread over all SMs first (consecutive items go to different blocks)
  const int back_blocks = (int)(ntot < c->num_sms ? ntot : c->num_sms);
  const int need_warps = (int)div_up(ntot, back_blocks);
  if (need_warps < back_warps) back_warps = need_warps;
  k_hh_back<<<back_blocks, back_warps * 32, (size_t)back_warps * zstride * sizeof(double2),
              c->stream>>>(a, zstride);
  note_launch(5);
  return cuda_check(c, cudaGetLastError(), "tridiagonal eigensolver");
}

// Eigendecomposition of np Hermitian matrices by the tridiagonal route, in
// groups whose work vectors fit in shared memory (problems of one group share
// every launch).  Returns SKY_EUNSUPPORTED, with nothing enqueued, when a
// single problem's vectors do not fit (or a device-gated batch would need more
// than one group); the caller then uses the Jacobi solver.
sky_status eigh_batch_tri(Ctx* c, int np, const double2* const* A, const int* n,
                          double* const* w, double2* const* Z, const int* run, int run_stride) {
  int groups[kMaxBatch + 1], order[kMaxBatch];
  bool gvec[kMaxBatch];
  int ng = 0;
  size_t used = 0;
  groups[0] = 0;
  if (np > kTeamMin) {
    // one launch sequence, the blocks split into teams (tri_group)
    for (int b = 0; b < np; ++b) {
      gvec[b] = false;
      order[b] = b;
      if (tri_vectors_global(n[b]) || n[b] > c->tri_m) return SKY_EUNSUPPORTED;
    }
    return tri_group(c, np, order, A, n, w, Z, run, run_stride, gvec);
  }
  // work vectors in global memory for problems too large for shared memory,
  // and, when the global buffer has room, for the largest problems until the
  // whole batch fits one launch sequence (a device-gated batch must: it
  // cannot be split)
  const bool room = c->d_trivec && np <= c->tri_vec_slots;
  size_t total = 0;
  for (int b = 0; b < np; ++b) {
    gvec[b] = tri_vectors_global(n[b]);
    total += ((gvec[b] ? 0 : 3 * (size_t)n[b]) + (n[b] + 1) / 2 + 1) * sizeof(double2);
  }
  while (room && total > kTriSmemMax) {
    int big = -1;
    for (int b = 0; b < np; ++b)
      if (!gvec[b] && (big < 0 || n[b] > n[big])) big = b;
    if (big < 0) break;
    gvec[big] = true;
    total -= 3 * (size_t)n[big] * sizeof(double2);
  }
  for (int b = 0; b < np; ++b) {
    const bool gv = gvec[b];
    if (gv && (!room || n[b] > c->tri_m)) return SKY_EUNSUPPORTED;
    const size_t need = ((gv ? 0 : 3 * (size_t)n[b]) + (n[b] + 1) / 2 + 1) * sizeof(double2);
    const size_t zneed = (size_t)(n[b] + (n[b] & 1)) * sizeof(double2);
    if (need > kTriSmemMax || zneed > kTriSmemMax) return SKY_EUNSUPPORTED;
    if (used + need > kTriSmemMax) {
      groups[++ng] = b;
      used = 0;
    }
    used += need;
    order[b] = b;
  }
  groups[++ng] = np;
  if (run && ng > 1) return SKY_EUNSUPPORTED;
  for (int g = 0; g < ng; ++g) {
    const sky_status s = tri_group(c, groups[g + 1] - groups[g], order + groups[g], A, n, w, Z,
                                   run, run_stride, gvec);
    if (s != SKY_OK) return s;
  }
  return SKY_OK;
}

}  // namespace sky
