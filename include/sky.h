/*
 * libsky: C ABI of the GB300 (sm_103a) damped-gradient Skyrme-DFT hot path
 * (Afibuzzaman, Schuetrumpf, Aktulga, arXiv 1610.07522).
 *
 * One iteration (Fig. 1, steps 2-5) is the sequence
 *   sky_apply_h(psi) -> sky_damped_step -> sky_apply_h(phi) -> sky_overlap (x2)
 *   -> sky_orthonormalize -> sky_subspace_diag -> sky_rotate
 *   -> sky_densities (per species) -> sky_mean_fields -> sky_energy,
 * with sky_sp_spread giving the convergence measure of Eq. convergence.
 *
 * Conventions shared by every entry point
 *   - All array arguments are DEVICE pointers owned by the caller.  No entry
 *     point frees or retains them past the call.
 *   - Every call is enqueued on the context's CUDA stream and returns without
 *     waiting.  The return value reports argument and launch errors.  Errors
 *     found on the device (SKY_ENOTPD, SKY_ENOCONV, SKY_ETIMEOUT, SKY_ENAN)
 *     are recorded in a device status word that sky_sync() returns and clears.
 *   - Grid: nx, ny, nz points with spacing dx (fm), periodic, x_a = a*dx.
 *     G = nx*ny*nz.  A spinor is 2 spin components of G points; V = 2G
 *     (Sec. 3.1, "psi(V,A)").
 *   - Spinor arrays: [I][2][nz][ny][nx] complex, x fastest, interleaved
 *     (re, im), in the context precision: double2 for SKY_F64, float2 for
 *     SKY_F32.  Consecutive states are V complex values apart.
 *   - Field arrays (rho, tau, divJ, U, B): [nz][ny][nx] double.  Vector
 *     fields (J, W): [3][nz][ny][nx] double, components x, y, z.
 *   - I x I matrices: row-major double2, element (a, b) at [a*I + b].
 *   - I must satisfy 0 <= I <= max_states given to sky_init; I == 0 is a no-op.
 *   - Units: MeV and fm.
 */
#ifndef SKY_H
#define SKY_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sky_ctx sky_ctx;

typedef enum {
  SKY_OK = 0,
  SKY_EINVAL = 1,       /* bad argument (null pointer, size out of range)        */
  SKY_ENOMEM = 2,       /* device allocation failed in sky_init                  */
  SKY_ECUDA = 3,        /* a CUDA runtime call or kernel launch failed           */
  SKY_ENOTPD = 4,       /* overlap matrix not positive definite (dependent phi)  */
  SKY_ENOCONV = 5,      /* Jacobi eigensolver hit its sweep limit                */
  SKY_ETIMEOUT = 6,     /* a bounded device-side wait gave up                    */
  SKY_ENAN = 7,         /* NaN or Inf in the energy                              */
  SKY_EUNSUPPORTED = 8  /* grid size or precision not built into this library   */
} sky_status;

typedef enum {
  SKY_F64 = 0,          /* complex double spinors, FP64 everywhere               */
  SKY_F32 = 1,          /* complex float spinors; matrices and sums FP64         */
  SKY_F32_BF16X3 = 2,   /* as SKY_F32, with the overlap and recombination on the
                           tensor cores: 2-way bf16 split, 3 products, FP32 sums */
  SKY_F32_BF16X6 = 3    /* as SKY_F32_BF16X3 with a 3-way split and 6 products   */
} sky_prec;

/* Skyrme parameters (Eq. Skyrme; the paper fits them without printing them).
 * t0 [MeV fm^3], t1, t2 [MeV fm^5], t3 [MeV fm^(3+3 alpha)], x0..x3, alpha,
 * W0 [MeV fm^5], hb2m_n/hb2m_p = hbar^2/2m [MeV fm^2], e2 = e^2 [MeV fm];
 * coulomb != 0 adds the FFT-Poisson Coulomb potential to the protons
 * (Sec. 2.2). */
typedef struct {
  double t0, t1, t2, t3;
  double x0, x1, x2, x3;
  double alpha, W0;
  double hb2m_n, hb2m_p, e2;
  int coulomb;
} sky_skyrme;

/* Create a context for one grid.  grid[3] = (nx, ny, nz), each from the sizes
 * sky_supported_size() accepts for the precision; dx[3] in fm; twist[3] is the
 * Bloch phase theta in [-pi, pi) per direction (NULL = 0), so derivatives use
 * k + theta/L; max_states bounds I in every later call and sizes the scratch
 * memory the context owns; stream is a cudaStream_t (NULL = legacy default
 * stream).  The device is the current CUDA device.  On success *out owns
 * device memory until sky_destroy.  Returns SKY_EINVAL / SKY_EUNSUPPORTED /
 * SKY_ENOMEM / SKY_ECUDA on failure with *out = NULL.  With the environment
 * variable SKY_FILL_SCRATCH_NAN=1, every device buffer a context allocates
 * (here or later) starts filled with 0xFF bytes, NaN in every floating-point
 * format: a check that no kernel reads scratch it has not written. */
sky_status sky_init(sky_ctx** out, const int grid[3], const double dx[3],
                    const sky_skyrme* params, const double twist[3],
                    sky_prec prec, int max_states, void* stream);

/* Free everything the context owns (waits for its stream first). */
sky_status sky_destroy(sky_ctx* ctx);

/* Change the stream later calls are enqueued on. */
sky_status sky_set_stream(sky_ctx* ctx, void* stream);

/* Wait for the context's stream; return and clear the device status word. */
sky_status sky_sync(sky_ctx* ctx);

/* Solver counters of the context (waits for its stream): out[0] Jacobi
 * eigensolves run, out[1] Jacobi sweeps in total, out[2] sweeps of the last
 * eigensolve, out[3] Loewdin factors computed, out[4] of them by the
 * Newton-Schulz route, out[5] Newton-Schulz iterations in total, out[6]
 * eigensolves by the tridiagonal route, out[7] reserved (0).  reset != 0
 * clears them afterwards. */
sky_status sky_stats(sky_ctx* ctx, long long out[8], int reset);

/* Human-readable text of the last error the context saw (never NULL). */
const char* sky_last_error(const sky_ctx* ctx);

/* Host <-> device copies on the context's stream, for callers whose state
 * lives in host memory (the paper's code keeps psi in host memory, Sec. 3.1):
 * sky_memcpy_h2d copies bytes from the HOST buffer src into the DEVICE buffer
 * dst, sky_memcpy_d2h from the DEVICE buffer src into the HOST buffer dst.
 * Enqueued (asynchronous with respect to the host for page-locked host
 * memory; pageable host memory makes the call wait for the copy); both
 * buffers stay owned by the caller and must stay valid until the stream has
 * run the copy.  SKY_ECUDA if the runtime rejects the copy. */
sky_status sky_memcpy_h2d(sky_ctx* ctx, void* dst, const void* src, size_t bytes);
sky_status sky_memcpy_d2h(sky_ctx* ctx, void* dst, const void* src, size_t bytes);

/* 1 if an axis of n points is built for precision prec, else 0. */
int sky_supported_size(int n, sky_prec prec);

/* Number of CUDA kernels this process has enqueued through libsky so far
 * (all contexts); for launch accounting by callers. */
unsigned long long sky_kernel_launches(void);

/* The team split the batched tridiagonal eigensolver uses for a batch of more
 * than 8 problems (Sec. 3.3.2; the blocks of its cooperative Householder
 * reduction split into teams with their own barriers): np problems of n[b]
 * states on `blocks` blocks (the GPU's SM count).  Writes team[b] (the team of
 * problem b), first[t] and count[t] (team t's blocks, contiguous, in order)
 * and returns the number of teams; 0 when the batch cannot be split (a
 * problem's work vectors exceed shared memory: the solver then takes Jacobi)
 * or an argument is invalid (np outside [1, 128], blocks < 1, n[b] < 1, null
 * pointers).  team holds np entries, first and count np each (at most np
 * teams).  Host only: needs no GPU and no context. */
int sky_tri_team_plan(int np, const int* n, int blocks, int* team, int* first, int* count);

/* ---- Step 2: single-particle Hamiltonian (Sec. 2.1-2.2, Eq. Schroedinger) --
 * hpsi = h psi for I states, h = U - sum_j d_j B d_j
 *        - (i/2) sum_ijk eps_ijk [W_i sigma_k d_j + d_j W_i sigma_k],
 * every derivative spectral along its axis with k + theta/L (Nyquist kept).
 * U, B: [G]; W: [3][G] (one species' mean field).  psi, hpsi: [I][2][G]
 * spinors, must not overlap.  eps (nullable, [I]) receives <psi|h|psi>,
 * hnorm2 (nullable, [I]) receives <h psi|h psi> (= <psi|h^2|psi>), both
 * with the volume element dx^3 (FP32 forms: sums of exact float products kept
 * in float pairs, about 2^-48 of the sum per term, totals in FP64).  Stored as
 * the paper's hampsi (Sec. 3.4). */
sky_status sky_apply_h(sky_ctx* ctx, const double* U, const double* B, const double* W,
                       const void* psi, void* hpsi, int I, double* eps, double* hnorm2);

/* ---- Spectral derivative along one axis (Sec. 2.2: the derivatives of the
 * method are taken with FFTs) ------------------------------------------------
 * dst = d_axis src for n arrays of G complex points each ([n][G], x fastest,
 * complex128 in the FP64 form, complex64 in the FP32 forms), with the
 * wavenumbers k + theta/L of the spinor derivatives (Nyquist kept): the
 * derivative every h psi and density call applies, one axis at a time
 * (axis 0 = x, 1 = y, 2 = z).  dst may equal src (in place), otherwise the
 * two must not overlap.  Arithmetic as SKY_KNOB_LINE_ARITH selects.
 * SKY_EINVAL for a bad axis, n < 0 or null pointers with n > 0. */
sky_status sky_derivative(sky_ctx* ctx, int axis, const void* src, void* dst, int n);

/* ---- Step 2: damped gradient step (Eq. dampstep) ---------------------------
 * phi = psi - x0 * P (hpsi - eps psi), P = 1/(E0 + hb2m_q |k + theta/L|^2)
 * diagonal in momentum space (hb2m_q of species q = 0 neutrons, 1 protons).
 * psi, hpsi, phi: [I][2][G]; phi must not overlap psi or hpsi; eps: [I].
 * x0 dimensionless step (the paper's delta), E0 in MeV.
 * w: NULL for the paper's step, or a device float [G] weight that scales
 * the update voxel by voxel, phi = psi - w(r) x0 P (hpsi - eps psi), the same
 * w for both spin components (e.g. from sky_net_forward).  Any w keeps the
 * fixed point, where (h - eps) psi = 0. */
sky_status sky_damped_step(sky_ctx* ctx, int q, const void* psi, const void* hpsi,
                           const double* eps, void* phi, int I, double x0, double E0,
                           const float* w);

/* ---- Time-dependent stepping (Sec. 2.2, the unitary time evolution of
 * Sky3D's time-dependent mode, Sec. 1) -----------------------------------------
 * out = sum_{k=0}^{order} (-i tau h)^k / k! psi, the Taylor polynomial of
 * the propagator exp(-i tau h) with tau = dt / hbar in MeV^-1 (dt in fm/c
 * divided by hbar c = 197.327 MeV fm) and h the single-particle Hamiltonian
 * of sky_apply_h with the mean field U, B, W of one species.  The states
 * need no orthonormalisation: the exact propagator is unitary and the
 * polynomial departs from it by the Taylor remainder |tau h|^(order+1) /
 * (order+1)!.  psi, out: [I][2][G]; work: device scratch of 2 I V complex
 * values in the context precision, owned by the caller and overwritten.
 * psi, out and work must not overlap; 0 <= order <= 32 (order 0 copies psi).
 * The mean field to pass (e.g. the one at the midpoint of the step) is the
 * caller's choice. */
sky_status sky_td_taylor(sky_ctx* ctx, const double* U, const double* B, const double* W,
                         const void* psi, void* out, void* work, int I, double tau, int order);

/* ---- Step 3a: overlap / Hamiltonian matrix (Eqs. normmatrix, hammatrix) ----
 * X[a*I + b] = <a_a | b_b> = dx^3 sum_v conj(a_a[v]) b_b[v] for a >= b, and
 * X[b*I + a] = conj(X[a*I + b]) (only the lower triangle is formed, Fig. 3).
 * S = sky_overlap(phi, phi), H = sky_overlap(phi, h phi).  X: [I*I]. */
sky_status sky_overlap(sky_ctx* ctx, const void* a, const void* b, int I, double* X);

/* ---- Step 3c: Loewdin orthonormalisation (Eqs. Loewedin, orthmatvec) ------
 * C = S^{-1/2} = X Lambda^{-1/2} X^H from the eigendecomposition of the
 * Hermitian overlap S [I*I].  C: [I*I], may not alias S.  A non-positive
 * eigenvalue sets SKY_ENOTPD on the device. */
sky_status sky_orthonormalize(sky_ctx* ctx, const double* S, int I, double* C);

/* ---- Steps 3b, 3d: diagonalisation and combination (Sec. 3.3.2-3.3.3) -----
 * Exact Rayleigh-Ritz in the Loewdin basis: H' = C^H H C = Z Lambda Z^H
 * (Lambda ascending), M = C Z.  H, C, M: [I*I]; eps: [I] receives Lambda.
 * The new states are psi_a = sum_b M[b*I + a] phi_b (sky_rotate). */
sky_status sky_subspace_diag(sky_ctx* ctx, const double* H, const double* C, int I,
                             double* M, double* eps);

/* ---- Steps 3b-3d for several independent species at once --------------------
 * The same operations as sky_orthonormalize and sky_subspace_diag for nb
 * problems (e.g. neutrons and protons, which interact only through the mean
 * field, Sec. 3.2, or the species of many independent boxes), solved together
 * in one batched launch sequence: one cooperative eigensolver launch serves
 * every problem.  1 <= nb <= the context's batch capacity (2 after sky_init,
 * see sky_reserve_batch); each I[b] <= max_states.  The matrices may belong
 * to other contexts' state sets: only their sizes matter here.  S, H, C, M,
 * eps, I are HOST arrays of nb entries, read during the call (so a captured
 * CUDA graph keeps the pointers it was captured with); the matrices they point
 * to are device memory as above. */
sky_status sky_orthonormalize_batched(sky_ctx* ctx, int nb, const double* const* S, const int* I,
                                      double* const* C);

/* The paper's combined form of steps 3b-3e (Sec. 3.3.3, Fig. step67), a
 * selectable variant: Z diagonalises H itself (the matrix of the
 * non-orthonormal states, H = Z Lambda Z^H, Lambda ascending into eps), and
 * the Loewdin factor C of the same states (from sky_orthonormalize*) is
 * applied after it, M = Z C, so that psi_a = sum_b M[b*I + a] phi_b
 * (sky_rotate).  M depends on the phases of Z's columns, which the paper
 * leaves open: each column's first component of largest modulus is made real
 * and positive (and for degenerate eigenvalues on the eigensolver's basis).  Equal to sky_subspace_diag when the states are orthonormal;
 * otherwise the new states are neither exactly orthonormal nor exact Ritz
 * vectors, a difference the paper notes vanishes at convergence.  Arguments
 * as sky_subspace_diag_batched. */
sky_status sky_subspace_diag_literal_batched(sky_ctx* ctx, int nb, const double* const* H,
                                             const double* const* C, const int* I,
                                             double* const* M, double* const* eps);

/* Raise the batch capacity of the batched calls to nb problems of up to
 * max_states each (1 <= nb <= 128).  Allocates device memory (about
 * 9.5 max_states^2 complex doubles per problem; for nb > 8 also the digit
 * buffers of the grouped tensor-core I x I products, about 72 max_states
 * bytes per problem and state plus partials, capped at 2 GiB each) and
 * synchronises the context stream; call it outside stream capture.
 * SKY_ENOMEM leaves the context as it was. */
sky_status sky_reserve_batch(sky_ctx* ctx, int nb);
sky_status sky_subspace_diag_batched(sky_ctx* ctx, int nb, const double* const* H,
                                     const double* const* C, const int* I, double* const* M,
                                     double* const* eps);

/* ---- Step 3e: recombination (Sec. 3.3.3, Fig. 3) ---------------------------
 * psi_out[a] = sum_b M[b*I + a] phi[b] for all V entries.  phi, psi_out:
 * [I][2][G] and must not overlap.  Also the Loewdin application of
 * Eq. orthmatvec when M = C. */
sky_status sky_rotate(sky_ctx* ctx, const void* phi, const double* M, int I, void* psi_out);

/* ---- Step 4a: densities (Eqs. rho, curr, tau; all v^2 = 1) -----------------
 * For the I states of one species: rho = sum |psi|^2, tau = sum |d psi|^2,
 * J_i = sum Re[-i eps_ijk psi^+ sigma_k d_j psi], divJ = sum_i d_i J_i
 * (spectral, real part).  rho, tau, divJ: [G]; J: [3][G] or NULL.  FP32 forms:
 * the sums over states of exact float products are kept in float pairs (about
 * 2^-48 of the sum per term), the splits added in FP64. */
sky_status sky_densities(sky_ctx* ctx, const void* psi, int I, double* rho, double* tau,
                         double* J, double* divJ);

/* ---- Step 4b: mean field (Eq. Skyrme, Sec. 2.2) ----------------------------
 * Both species at once (the only neutron-proton coupling, Sec. 3.2).
 * rho, tau, divJ: [2][G] (neutrons then protons).  U, B: [2][G]; W: [2][3][G].
 * U_q = dE/drho_q (Coulomb added to protons when enabled), B_q = dE/dtau_q,
 * W_q = dE/dJ_q of the isoscalar/isovector Skyrme functional. */
sky_status sky_mean_fields(sky_ctx* ctx, const double* rho, const double* tau,
                           const double* divJ, double* U, double* B, double* W);

/* ---- Step 5: energy (Eq. Skyrme; Coulomb by FFT Poisson) -------------------
 * out[8] (device doubles): total E, kinetic, rho^2 (+density dependent),
 * rho tau, rho Delta rho, rho div J, Coulomb, particle number A = int rho.
 * A NaN or Inf total sets SKY_ENAN. */
sky_status sky_energy(sky_ctx* ctx, const double* rho, const double* tau,
                      const double* divJ, double* out);

/* ---- Step 5: convergence measure (Eq. convergence) -------------------------
 * out[0] = sqrt( sum_a (hnorm2[a] - eps[a]^2) / A ), out[1] = sum_a eps[a],
 * over A states (pass both species' arrays back to back). */
sky_status sky_sp_spread(sky_ctx* ctx, const double* eps, const double* hnorm2, int A,
                         double* out);

/* ---- Precision form of a running context -------------------------------------
 * Switch an FP32-spinor context among SKY_F32, SKY_F32_BF16X3 and
 * SKY_F32_BF16X6 (the spinor storage stays complex FP32; only the overlap and
 * recombination change).  A solver may run the cheap split-BF16 form while
 * far from convergence and finish in a more accurate one, since the BF16
 * forms' orthonormality error (about 1e-5 for x3) bounds how close they can
 * get to the FP64 fixed point.  Switching to a split-BF16 form may allocate
 * its operand pieces (and synchronises the context stream): call it outside
 * stream capture.  An FP64 context cannot switch (SKY_EUNSUPPORTED). */
sky_status sky_set_prec(sky_ctx* ctx, sky_prec prec);

/* ---- Tunable launch shapes ---------------------------------------------------
 * Launch-shape knobs of a context, for an autotuner that times the calls on
 * its own workload and keeps the fastest values, and two limits of the
 * device-side waits and iterations.  Every value gives the same
 * result except for the order of floating-point sums (split counts, eigensolver
 * blocks), so results may change in the last bits.  The paper has no
 * counterpart (its tuning is the MPI/OpenMP layout, Sec. 5).
 *   SKY_KNOB_LINE_YZ        threads per block of the y/z FFT line passes: 32, 64, 128
 *   SKY_KNOB_LINE_X         lines per block of the x FFT line passes: 16, 32, 64
 *   SKY_KNOB_OVERLAP_WAVES  FMA overlap: K splits filling 1 or 2 waves of blocks
 *   SKY_KNOB_TC_WAVES       split-BF16 overlap: K splits filling 1, 2 or 4 waves of SMs,
 *                           or 0: the fewest splits the FP32 accumulation bound allows
 *                           (2048 values of K each; for contexts that share the GPU with
 *                           other boxes' work)
 *   SKY_KNOB_TC_TILE_N      split-BF16 overlap and recombination GEMM tiles: 128 x 256
 *                           (256), 128 x 128 (128) or 0 (default: 256 for x3 when N allows)
 *   SKY_KNOB_FUSED_H        FP32 forms with every axis length in {8, 12, 16, 20, 24, 32}:
 *                           1 applies h psi in one pass per axis (each line's derivative,
 *                           spin-orbit and flux terms and the flux derivative in registers,
 *                           h psi read and written once per pass), 0 the general gradient /
 *                           local / divergence passes; default 1 when every axis is at most
 *                           24, else 0
 *   SKY_KNOB_JACOBI_BLOCKS  blocks of the cooperative eigensolver: 1..JACOBI_BLOCKS_MAX
 *                           (until set: one per SM, two per SM for problems >= 512)
 *   SKY_KNOB_JACOBI_BLOCKS_MAX  (read only) co-resident blocks of that kernel
 *   SKY_KNOB_WAIT_SPINS     spin budget of each grid-barrier wait of the eigensolver, in
 *                           thousands of tries (default 40000, i.e. about a second); a wait
 *                           that runs out sets SKY_ETIMEOUT and the kernel returns, leaving
 *                           the context usable (0 makes every wait give up at once)
 *   SKY_KNOB_JACOBI_MAX_SWEEPS  Jacobi sweeps before SKY_ENOCONV (1..1000, default 60)
 *   SKY_KNOB_EIGEN_METHOD   the FP64 eigensolver behind every diagonalisation:
 *                           SKY_EIG_JACOBI (parallel cyclic Jacobi), SKY_EIG_TRIDIAGONAL
 *                           (Householder reduction to real tridiagonal form, bisection,
 *                           inverse iteration, back-transformation: the paper's route
 *                           through ScaLAPACK, Sec. 3.3.2) or SKY_EIG_AUTO (default:
 *                           tridiagonal for batches with a problem of 64 states or more,
 *                           Jacobi for batches of smaller problems only; a batch of more
 *                           than 8 problems splits the reduction's blocks into teams, one
 *                           per large problem and shared ones for small problems; the
 *                           tridiagonal route falls back to Jacobi when its work vectors
 *                           exceed shared memory)
 *   SKY_KNOB_SPLIT_GEMM     FP64 and FP32 forms: 1 (default) computes sky_overlap and
 *                           sky_rotate on the tensor cores as exact-integer split products
 *                           (each row scaled by a power of two and cut into signed 8-bit
 *                           digits held exactly in bf16: 6 digits and 21 digit products for
 *                           SKY_F64, 4 and 10 for SKY_F32; every digit product summed
 *                           exactly in FP32 over segments of 128 values of K, the segments
 *                           added in pairs of FP32 by error-free transformations), about
 *                           1e-14 (FP64) and 1e-9 (FP32) of the largest result; 0 runs the
 *                           FP64 FMA kernels on the CUDA cores.  Switching to 1 may allocate
 *                           the digit buffers; not allowed for the split-BF16 forms
 *   SKY_KNOB_LINE_ARITH     FP64 form, the spectral derivatives of h psi and the densities
 *                           (Sec. 2.2): 2 (default) applies each axis's derivative as the
 *                           dense circulant operator of the FFT form, a product of six-digit
 *                           exact-integer splits of the lines and of the operator on the
 *                           tensor cores (about 2^-48 of the line's largest value, rounded
 *                           once to FP64); 1 runs the FFT line passes in double-float
 *                           arithmetic (pairs of FP32 values, about 48 significant bits;
 *                           GB300 issues FP32 operations at about 77x its FP64 rate); 0 runs
 *                           them in FP64.  2 needs axis lengths in {8, 12, 16, 20, 24, 32}
 *                           (the lengths the FP64 form accepts).  The FP32 forms accept 0 only
 * sky_tune_set returns SKY_EINVAL for a value outside these sets; sky_tune_get
 * returns the current value (-1 for an unknown knob or a NULL context). */
typedef enum {
  SKY_KNOB_LINE_YZ = 0,
  SKY_KNOB_LINE_X = 1,
  SKY_KNOB_OVERLAP_WAVES = 2,
  SKY_KNOB_TC_WAVES = 3,
  SKY_KNOB_JACOBI_BLOCKS = 4,
  SKY_KNOB_JACOBI_BLOCKS_MAX = 5,
  SKY_KNOB_WAIT_SPINS = 6,
  SKY_KNOB_JACOBI_MAX_SWEEPS = 7,
  SKY_KNOB_EIGEN_METHOD = 8,
  SKY_KNOB_SPLIT_GEMM = 9,
  SKY_KNOB_LINE_ARITH = 10,
  SKY_KNOB_TC_TILE_N = 11,
  SKY_KNOB_FUSED_H = 12
} sky_knob;
enum { SKY_EIG_AUTO = 0, SKY_EIG_JACOBI = 1, SKY_EIG_TRIDIAGONAL = 2 };
sky_status sky_tune_set(sky_ctx* ctx, sky_knob knob, int value);
int sky_tune_get(const sky_ctx* ctx, sky_knob knob);

/* ---- Learned damping weight ----------------------------------------------
 * The paper has no learned part; these calls build and train a per-voxel
 * weight w_q(r) for the damped step of Eq. dampstep (sky_damped_step's w).
 * Network: three periodic 3x3x3 cross-correlations,
 *   x  = (U_q / SKY_NET_USCALE, B_q / hb2m_q - 1, |W_q| / SKY_NET_WSCALE)
 *   h1 = tanh(conv(x; W1, b1)), h2 = tanh(conv(h1; W2, b2)),
 *   w  = SKY_NET_WMAX * sigmoid(conv(h2; W3, b3)),
 * conv(x; W, b)_o(r) = b_o + sum_i sum_d W[o][i][t] x_i(r + d) over
 * d in {-1, 0, 1}^3 with t = 9 (dz+1) + 3 (dy+1) + (dx+1).
 * theta: device float [SKY_NET_NPARAM] = W1 [16][3][27], b1 [16],
 * W2 [16][16][27], b2 [16], W3 [1][16][27], b3 [1].
 * ws: device float workspace [SKY_NET_WS_PER_POINT * G], owned by the caller;
 * sky_net_backward reads the activations the previous sky_net_forward on the
 * same ws left there.  Everything is FP32 except the loss, the statistics and
 * the gradients (FP64); all sums are in a fixed order (deterministic). */
#define SKY_NET_HIDDEN 16
#define SKY_NET_NPARAM 8673
#define SKY_NET_WS_PER_POINT 69
#define SKY_NET_WMAX 4.0
#define SKY_NET_USCALE 50.0
#define SKY_NET_WSCALE 5.0

/* The network's weight w_net [G] from the mean field of species q (U, B: [G];
 * W: [3][G], the arrays sky_apply_h takes) is kept in ws; w receives the
 * weight the step uses, w = 1 + scale (w_net - 1), scale in [0, 1] (1: the
 * network's own weight, 0: the paper's step; a solver may lower it when the
 * energy rises). */
sky_status sky_net_forward(sky_ctx* ctx, int q, const float* theta, const double* U,
                           const double* B, const double* W, double scale, float* ws, float* w);

/* Loss L = sum_r (a w_net^2 - 2 b w_net + c) / norm of one training sample,
 * where abc = [a; b; c] ([3][G] double) and norm (device double [1]) come
 * from sky_precond_stats and w_net is the network weight the last
 * sky_net_forward left in ws.  Adds L to loss[0] and dL/dtheta to grad
 * [SKY_NET_NPARAM] (both device doubles, accumulated so that several
 * samples sum). */
sky_status sky_net_backward(sky_ctx* ctx, const float* theta, float* ws, const double* abc,
                            const double* norm, double* grad, double* loss);

/* One Adam step (Kingma and Ba, 2015) on theta with the moment estimates m, v
 * (device doubles [SKY_NET_NPARAM], zero before step 1); step counts from 1.
 * Sets grad to zero after using it. */
sky_status sky_net_adam(sky_ctx* ctx, float* theta, double* grad, double* m, double* v, int step,
                        double lr, double beta1, double beta2, double eps);

/* Full cross overlap X[a*I + b] = <a_a | b_b> = dV sum_v conj(a_a[v]) b_b[v]
 * of two different state sets (no Hermitian mirror), FP64 accumulation in
 * every precision.  a, b: [I][2][G]; X: [I*I] double2.  With a = psi* and
 * b = psi, sky_rotate(psi*, X) gives the projection of psi on span(psi*). */
sky_status sky_cross_overlap(sky_ctx* ctx, const void* a, const void* b, int I, double* X);

/* Per-voxel statistics of the one-step loss for one species:
 *   a(r) = sum |psi - phi|^2,  b(r) = sum Re(conj(psi - phi)(psi - ppsi)),
 *   c(r) = sum |psi - ppsi|^2  (sums over the I states and both spins),
 * with phi the plain damped step of psi (w = NULL) and ppsi the projection
 * of psi on the converged occupied space.  abc: [3][G] double; norm[0] =
 * sum_r c(r).  psi, phi, ppsi: [I][2][G] in the context precision. */
sky_status sky_precond_stats(sky_ctx* ctx, const void* psi, const void* phi, const void* ppsi,
                             int I, double* abc, double* norm);

/* ---- Overlap matrix without a context or any device allocation -----------
 * The paper has no counterpart to this entry point.  It computes the same
 * matrix as sky_overlap, X[a*I + b] = dV * sum_v conj(a_a[v]) b_b[v] (lower
 * triangle formed, mirrored), for callers that are not allowed to allocate
 * device memory -- e.g. code inside a host application whose allocator owns
 * the whole device-memory budget -- and so cannot create a context.
 * a, b: [I][V] complex in precision prec (double2 or float2); X: [I*I]
 * double2, all device pointers owned by the caller; V complex entries per
 * state; dV the volume element; stream a cudaStream_t (NULL = default).
 * Its scratch is one fixed 16 MiB device array inside the library, held by
 * every GPU that loads it until exit; I is limited to 1024 (SKY_EINVAL
 * above).  Every call looks the array's address up in the CUDA context
 * current at the call (so a device reset or another context on the device
 * gets its own copy); the first call in a context loads the library's device
 * code there and should come before any stream capture.  Calls share the
 * array: calls that overlap in time on the GPU race.  If a CUDA error is
 * already pending when the call starts, it returns SKY_ECUDA without work and
 * leaves that error for the caller.  Calls no cudaMalloc or cudaFree. */
sky_status sky_overlap_noalloc(const void* a, const void* b, int I, long long V, double dV,
                               sky_prec prec, double* X, void* stream);

/* ---- FMA-rate probe -----------------------------------------------------------
 * The paper has no counterpart: a measurement aid for roofline fractions.
 * Enqueues one kernel of blocks_per_sm (1..64) blocks of 256 threads per SM on
 * stream, each thread running 8 independent FMA chains for iters (>= 1)
 * iterations in FP64 (fp64 != 0) or FP32, and sets *flops (host) to the
 * floating-point operations it executes (2 per FMA).  Time it with events on
 * the same stream: flops / time is the device's FMA rate in that precision.
 * Allocates nothing and writes no device memory. */
sky_status sky_fma_probe(int fp64, int blocks_per_sm, int iters, void* stream, double* flops);

#ifdef __cplusplus
}
#endif
#endif /* SKY_H */
