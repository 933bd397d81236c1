// Internal definitions shared by the libsky translation units: complex
// helpers, the context structure, status plumbing and launch helpers.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <cstdio>
#include <type_traits>

#include "sky.h"

namespace sky {

// ----------------------------------------------------------------- complex
template <typename T> struct CxT;
template <> struct CxT<double> { using type = double2; };
template <> struct CxT<float> { using type = float2; };
template <typename T> using cx = typename CxT<T>::type;

template <typename T> __host__ __device__ __forceinline__ cx<T> mkc(T a, T b) {
  cx<T> r; r.x = a; r.y = b; return r;
}
#define SKY_CX_OPS(V, S)                                                              \
  __host__ __device__ __forceinline__ V operator+(V a, V b) { V r; r.x = a.x + b.x; r.y = a.y + b.y; return r; } \
  __host__ __device__ __forceinline__ V operator-(V a, V b) { V r; r.x = a.x - b.x; r.y = a.y - b.y; return r; } \
  __host__ __device__ __forceinline__ V operator-(V a) { V r; r.x = -a.x; r.y = -a.y; return r; }              \
  __host__ __device__ __forceinline__ V operator*(S s, V a) { V r; r.x = s * a.x; r.y = s * a.y; return r; }    \
  __host__ __device__ __forceinline__ V cmul(V a, V b) { V r; r.x = a.x * b.x - a.y * b.y; r.y = a.x * b.y + a.y * b.x; return r; } \
  __host__ __device__ __forceinline__ V cmulc(V a, V b) { V r; r.x = a.x * b.x + a.y * b.y; r.y = a.x * b.y - a.y * b.x; return r; } \
  __host__ __device__ __forceinline__ V conjx(V a) { V r; r.x = a.x; r.y = -a.y; return r; }                   \
  __host__ __device__ __forceinline__ V mul_i(V a) { V r; r.x = -a.y; r.y = a.x; return r; }                    \
  __host__ __device__ __forceinline__ V mul_mi(V a) { V r; r.x = a.y; r.y = -a.x; return r; }
SKY_CX_OPS(double2, double)
SKY_CX_OPS(float2, float)
#undef SKY_CX_OPS
// cmulc(a, b) = conj(a) * b.

__device__ __forceinline__ double2 to_d2(double2 a) { return a; }
__device__ __forceinline__ double2 to_d2(float2 a) { return make_double2(a.x, a.y); }
template <typename T> __device__ __forceinline__ cx<T> from_d2(double2 a);
template <> __device__ __forceinline__ double2 from_d2<double>(double2 a) { return a; }
template <> __device__ __forceinline__ float2 from_d2<float>(double2 a) {
  return make_float2((float)a.x, (float)a.y);
}

// ----------------------------------------------------------------- context
// Isoscalar (index 0) / isovector (index 1) Skyrme couplings, host-computed.
struct Couplings {
  double rho[2], rhoa[2], tau[2], drho[2], nJ[2];
  double alpha, hb2m[2], e2;
  int coulomb;
};

struct Ctx;  // defined below; sky_ctx is an alias at the C boundary

constexpr int kDensSplits = 8;     // state splits of the density accumulation
constexpr int kMaxBatch = 128;     // problems per batched eigensolve / small GEMM
constexpr int kRedBlock = 256;     // threads of the per-state reduction blocks
constexpr int kMaxOverlapWaves = 2; // largest tunable K-split wave count of k_overlap
constexpr long long kBarrierSpins = 40000000;  // default spins (~32 ns each) per barrier wait
constexpr int kJacMaxSweeps = 60;   // default Jacobi sweep cap
constexpr int kMaxTcWaves = 4;      // largest tunable K-split wave count of the tcgen05 overlap

struct Ctx {
  // geometry
  int n[3];
  double dx[3], L[3], theta[3];
  int G;
  double dV;
  sky_prec prec;
  int max_states;
  int csize;            // bytes per complex spinor entry
  Couplings cp;
  cudaStream_t stream;
  int device, num_sms;
  // device memory owned by the context
  int* d_status;                    // device status word (sky_status bits)
  double* d_kt[3];                  // twisted wavenumbers k + theta/L (FP64)
  float* d_ktf[3];                  // the same in FP32
  double* d_kp[3];                  // plain wavenumbers (real fields)
  float2* d_ktdd[3];                // (k + theta/L) / n as float pairs (double-float passes)
  int line_arith;                   // FP64 derivative passes: 0 FP64 FFT, 1 double-float FFT,
                                    // 2 digit-split operator on the tensor cores
  void* d_dop[3];                   // tensor-core derivative operators: digits, smem layout
  int* d_dope[3];                   // their row exponents
  void* d_dft[3][2];                // forward / inverse DFT operators of each axis (same form)
  int* d_dfte[3][2];
  double* d_damp[2];                // 1 / (E0 + hb2m_q |k + theta/L|^2), [G]
  double damp_E0[2];                // E0 the tables were built for (NaN = none)
  double* d_coul;                   // 4 pi e^2 / |k|^2 (0 at k = 0), [G]
  void* d_gscr;                     // derivative scratch: 3 * chunk * V complex
  int chunk;                        // states per apply_h / densities chunk
  double* d_red;                    // per-state partial sums [max_states][nblk][2]
  int red_nblk;                     // reduction blocks per state
  double* d_dpart;                  // density partials [kDensSplits][5][G]
  double* d_ftmp;                   // field temporaries [16][G]
  double2* d_fcx;                   // complex field scratch [G]
  float* d_hf;                      // FP32 forms: U, B, W of one species as floats [5][G]
  int fused_h;                      // FP32 forms: one fused pass per axis for h psi (tunable)
  double2* d_gpart;                 // split-K partials of sky_overlap
  size_t gpart_elems;
  int ov_slots;                     // resident CTAs of the overlap kernel
  double2* d_eigA[2];               // Jacobi ping-pong matrices [m*m]
  double2* d_eigV;                  // Jacobi rotations accumulated [m*m]
  double* d_eigw;                   // eigenvalues [m]
  double* d_eigpart;                // per-block partial norms
  unsigned* d_bar;                  // grid barrier {count, generation}
  unsigned* d_tbar;                 // team barrier counters of the tridiagonal reduction
  int* d_eigres;                    // which ping-pong buffer holds each result [kMaxBatch]
  int eig_batch;                    // problems a batched eigensolve may hold
  size_t eig_slot;                  // elements per problem in d_eigA / d_eigV
  size_t eig_slot_rot;              // rotations per problem and round buffer
  size_t small_slot;                // elements per problem in each d_small buffer
  void* d_eigrot;                   // Jacobi rotations of two consecutive rounds
  int eig_grid;                     // blocks of the Jacobi kernel (tunable, <= eig_grid_max)
  int eig_grid_max;                 // co-resident blocks of the Jacobi kernel
  bool eig_grid_auto;               // eig_grid not tuned: chosen per solve from the size
  int line_yz;                      // threads per block of the y/z line passes (tunable)
  int line_x;                       // lines per block of the x line passes (tunable)
  int ov_waves;                     // K-split waves of the FMA overlap (tunable)
  long long wait_spins;             // spin budget of the eigensolver's grid-barrier waits
  int jac_max_sweeps;               // Jacobi sweeps before SKY_ENOCONV
  int tc_waves;                     // K-split waves of the tensor-core overlap (tunable)
  int tc_tile_n;                    // N width of the split-BF16 GEMM tiles: 0 auto, 128, 256
  double2* d_small[6];              // I x I temporaries
  void* d_tcA[3];                   // split-BF16 operand pieces (tensor-core forms)
  void* d_tcB[3];
  void* d_tcRotA[3];
  float* d_tcPart;                  // split-K partial tiles of the tensor-core overlap
  size_t tc_partial_elems;
  int* d_gate;                      // device-side gates of the Loewdin paths [8]
  long long* d_stats;               // solver counters reported by sky_stats [8]
  double* d_netpart;                // partial sums of the damping-network kernels
  int eig_method;                   // SKY_EIG_AUTO / SKY_EIG_JACOBI / SKY_EIG_TRIDIAGONAL
  double* d_trid;                   // tridiagonal solver vectors and LU rows [tri_slot] per problem
  size_t tri_slot;                  // doubles per problem in d_trid
  int tri_m;                        // vector stride inside a d_trid slot (even)
  double2* d_trivec;                // per-block work vectors of problems too large for shared memory
  int tri_vec_slots;                // problems d_trivec has room for
  // exact-integer split GEMMs of the FP64 and FP32 forms (oz_ops.cu)
  int oz_on;                        // 1: tensor-core split GEMMs, 0: FP64 FMA kernels
  void* d_ozA;                      // bf16 slices of the row operand
  void* d_ozB;                      // bf16 slices of the column operand
  int* d_ozE;                       // row exponents
  float2* d_ozP;                    // split-K partials (hi, lo)
  size_t oz_a_elems, oz_b_elems, oz_p_elems;
  // grouped I x I products of a batched eigensolve (oz_zgemm_group): digits of
  // up to ozg_rows stacked rows (A; B twice as many) of row stride ozg_ld,
  // partials, row exponents; allocated by sky_reserve_batch for batches of
  // more than kOzGroupMin problems
  void* d_ozgA;
  void* d_ozgB;
  float2* d_ozgP;
  int* d_ozgE;
  int ozg_rows, ozg_np;
  long long ozg_ld;
  size_t ozg_p_elems;
  char err[256];
};

// ----------------------------------------------------------------- status
#define SKY_STATUS_BIT(s) (1 << (int)(s))

__device__ __forceinline__ void flag_status(int* st, sky_status s) {
  atomicOr(st, SKY_STATUS_BIT(s));
}

sky_status set_err(Ctx* c, sky_status s, const char* fmt, ...);
sky_status cuda_check(Ctx* c, cudaError_t e, const char* what);

// Process-wide count of kernels enqueued by the library.
void note_launch(unsigned n = 1);

inline unsigned div_up(long long a, long long b) { return (unsigned)((a + b - 1) / b); }

// Host-side entry points of the other translation units.
sky_status upload_twiddles_hamiltonian(Ctx* c);
sky_status upload_twiddles_fields(Ctx* c);
sky_status apply_h_impl(Ctx* c, const double* U, const double* B, const double* W,
                        const void* psi, void* hpsi, int I, double* eps, double* hn2);
sky_status td_taylor_impl(Ctx* c, const double* U, const double* B, const double* W,
                          const void* psi, void* out, void* work, int I, double tau, int order);
sky_status damped_step_impl(Ctx* c, int q, const void* psi, const void* hpsi,
                            const double* eps, void* phi, int I, double x0, double E0,
                            const float* w);
sky_status densities_impl(Ctx* c, const void* psi, int I, double* rho, double* tau,
                          double* J, double* divJ);
sky_status mean_fields_impl(Ctx* c, const double* rho, const double* tau,
                            const double* divJ, double* U, double* B, double* W);
sky_status energy_impl(Ctx* c, const double* rho, const double* tau, const double* divJ,
                       double* out);
sky_status sp_spread_impl(Ctx* c, const double* eps, const double* hn2, int A, double* out);
sky_status overlap_impl(Ctx* c, const void* a, const void* b, int I, double2* X);
sky_status rotate_impl(Ctx* c, const void* phi, const double2* M, int I, void* out);
sky_status cross_overlap_impl(Ctx* c, const void* a, const void* b, int I, double2* X);
size_t net_partial_elems(int G);
sky_status net_forward_impl(Ctx* c, int q, const float* theta, const double* U, const double* B,
                            const double* W, double scale, float* ws, float* w);
sky_status net_backward_impl(Ctx* c, const float* theta, float* ws, const double* abc,
                             const double* norm, double* grad, double* loss);
sky_status net_adam_impl(Ctx* c, float* theta, double* grad, double* m, double* v, int step,
                         double lr, double beta1, double beta2, double eps);
sky_status precond_stats_impl(Ctx* c, const void* psi, const void* phi, const void* ppsi, int I,
                              double* abc, double* norm);
struct ZJobs {
  const double2* A[kMaxBatch];
  const double2* B[kMaxBatch];
  double2* C[kMaxBatch];
  int n[kMaxBatch];
  const int* run[kMaxBatch];
  const int* stop[kMaxBatch];
  int np;
  bool ah, bh;
};
ZJobs zjobs(int np, bool ah, bool bh, const double2* const* A, const double2* const* B,
            double2* const* C, const int* n, const int* const* run, const int* const* stop);
sky_status zgemm_batch(Ctx* c, const ZJobs& j);
sky_status zgemm_small(Ctx* c, bool ah, bool bh, const double2* A, const double2* B,
                       double2* C, int n, const int* run = nullptr, const int* stop = nullptr);
sky_status eigh_batch(Ctx* c, int np, const double2* const* A, const int* n, double* const* w,
                      double2* const* Z, const int* run, int run_stride);
sky_status lowdin_batch(Ctx* c, int np, const double2* const* S, const int* I, double2* const* C);
sky_status subspace_batch(Ctx* c, int np, const double2* const* H, const double2* const* C,
                          const int* I, double2* const* M, double* const* eps);
sky_status subspace_literal_batch(Ctx* c, int np, const double2* const* H,
                                  const double2* const* C, const int* I, double2* const* M,
                                  double* const* eps);
sky_status eigh_batch_tri(Ctx* c, int np, const double2* const* A, const int* n,
                          double* const* w, double2* const* Z, const int* run, int run_stride);
sky_status tri_init(Ctx* c);
// Derivative passes of the FP64 form as digit-split operator products on the
// tensor cores (oz_deriv.cu): operators built at context creation for axis
// lengths 8, 12, 16, 20, 24, 32; dst = d_ax src over nb arrays (dst may be src).
sky_status derivative_impl(Ctx* c, int axis, const void* src, void* dst, int n);
sky_status deriv_tc_init(Ctx* c);
cudaError_t deriv_tc(Ctx* c, int ax, const double2* src, double2* dst, long long nb);
bool damp_tc_available(const Ctx* c);
cudaError_t damp_tc(Ctx* c, int q, const double2* psi, const double2* hpsi, const double* eps,
                    double2* phi, int I, double x0, const float* w);
bool tri_vectors_global(int n);
size_t tri_vec_elems(int m, int nb, int nsm);
inline size_t tri_slot_doubles(int m) { return (size_t)m * m + 18 * (size_t)m; }
sky_status eigh_impl(Ctx* c, const double2* A, int I, double* w, double2* Z,
                     const int* run = nullptr);
sky_status lowdin_impl(Ctx* c, const double2* S, int I, double2* C);
sky_status subspace_impl(Ctx* c, const double2* H, const double2* C, int I, double2* M,
                         double* eps);
int jacobi_max_grid(Ctx* c);
int tc_nsplit(sky_prec p);
void tc_scratch_sizes(int I, long long V, int num_sms, size_t* piece_a, size_t* piece_b,
                      size_t* piece_rot_a, size_t* partial);
sky_status tc_overlap(Ctx* c, const void* a, const void* b, int I, double2* X);
void oz_scratch_sizes(sky_prec prec, int Imax, long long V, int nsm, size_t* a_elems,
                      size_t* b_elems, size_t* e_elems, size_t* p_elems);
sky_status oz_overlap(Ctx* c, const void* a, const void* b, int I, double2* X);
sky_status oz_rotate(Ctx* c, const void* phi, const double2* M, int I, void* out);
// I x I complex products from this many states on go to the tensor cores;
// device-gated ones (the Newton-Schulz iterations, most of which the device
// skips) from kOzZgemmGated on: a skipped product still enqueues the
// digit-split launch sequence (four short launches), which at 24^3 with
// 280 + 120 states costs less than the FP64 products it replaces (19.9 ms
// per iteration against 20.0 with the threshold at 768); ungated products
// of 96 states and more (120 x 120: 75 us as FP64 3M products, less on the
// tensor cores) take the tensor cores too (19.81 ms)
constexpr int kOzZgemmMin = 96;
constexpr int kOzZgemmGated = 192;
bool oz_zgemm_fits(const Ctx* c, int n);
bool oz_zgemm_group_fits(const Ctx* c, int np, const int* n);
sky_status oz_zgemm_group(Ctx* c, const ZJobs& j);
int oz_group_slices();
bool fused_h_ok(const Ctx* c);      // the fused FP32 h psi applies to this context
int tri_team_plan(int np, const int* n, int blocks, int* team, int* first, int* count);
int fused_h_blocks(const Ctx* c);   // its reduction blocks per state               // digits of the grouped products
constexpr int kOzGroupMin = 8;      // batches of more problems take the grouped products
sky_status oz_zgemm(Ctx* c, bool ah, bool bh, const double2* A, const double2* B, double2* C,
                    int n, const int* run, const int* stop);
sky_status tc_rotate(Ctx* c, const void* phi, const double2* M, int I, void* out);
inline bool is_tc(sky_prec p) { return p == SKY_F32_BF16X3 || p == SKY_F32_BF16X6; }
size_t jacobi_rot_bytes(int m);
size_t overlap_partial_elems(int I, long long V, int slots);
int overlap_slots(int num_sms);

}  // namespace sky

struct sky_ctx : public sky::Ctx {};
