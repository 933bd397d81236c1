// C ABI of libsky: context creation (wavenumber tables, scratch sized for
// max_states), argument checks and dispatch to the kernels.
#include <cmath>
#include <cstdarg>
#include <cstdlib>
#include <cstring>
#include <atomic>
#include <new>

#include "sky_internal.cuh"

namespace sky {

sky_status set_err(Ctx* c, sky_status s, const char* fmt, ...) {
  if (c) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(c->err, sizeof(c->err), fmt, ap);
    va_end(ap);
  }
  return s;
}

sky_status cuda_check(Ctx* c, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return SKY_OK;
  return set_err(c, SKY_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

sky_status build_coulomb_table(Ctx* c);   // fields.cu

static bool size_ok(int n, sky_prec p) {
  switch (n) {
    case 8: case 12: case 16: case 20: case 24: case 32: return true;
    case 48: case 64: return p != SKY_F64;
    default: return false;
  }
}

static Couplings couplings(const sky_skyrme& p) {
  Couplings c;
  c.rho[0] = 3.0 * p.t0 / 8.0;
  c.rho[1] = -p.t0 * (0.5 + p.x0) / 4.0;
  c.rhoa[0] = p.t3 / 16.0;
  c.rhoa[1] = -p.t3 * (0.5 + p.x3) / 24.0;
  c.tau[0] = 3.0 * p.t1 / 16.0 + p.t2 * (1.25 + p.x2) / 4.0;
  c.tau[1] = -p.t1 * (0.5 + p.x1) / 8.0 + p.t2 * (0.5 + p.x2) / 8.0;
  c.drho[0] = -9.0 * p.t1 / 64.0 + p.t2 * (1.25 + p.x2) / 16.0;
  c.drho[1] = 3.0 * p.t1 * (0.5 + p.x1) / 32.0 + p.t2 * (0.5 + p.x2) / 32.0;
  c.nJ[0] = -0.75 * p.W0;
  c.nJ[1] = -0.25 * p.W0;
  c.alpha = p.alpha;
  c.hb2m[0] = p.hb2m_n;
  c.hb2m[1] = p.hb2m_p;
  c.e2 = p.e2;
  c.coulomb = p.coulomb;
  return c;
}

// SKY_FILL_SCRATCH_NAN=1 in the environment: every buffer a context allocates
// starts as 0xFF bytes (NaN in every floating-point format), so a kernel that
// reads scratch it has not written shows up as NaN in the results.
static bool fill_nan() {
  const char* s = getenv("SKY_FILL_SCRATCH_NAN");
  return s && s[0] == '1';
}

template <typename T>
static sky_status dalloc(Ctx* c, T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
  if (e == cudaSuccess && fill_nan()) e = cudaMemset(*p, 0xFF, count * sizeof(T));
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return set_err(c, SKY_ENOMEM, "cudaMalloc of %zu bytes failed", count * sizeof(T));
  }
  return SKY_OK;
}

static void free_all(Ctx* c) {
  void* ptrs[] = {c->d_status, c->d_kt[0], c->d_kt[1], c->d_kt[2], c->d_ktdd[0], c->d_ktdd[1],
                  c->d_ktdd[2], c->d_ktf[0], c->d_ktf[1],
                  c->d_ktf[2], c->d_kp[0], c->d_kp[1], c->d_kp[2], c->d_damp[0], c->d_damp[1],
                  c->d_coul, c->d_gscr, c->d_red, c->d_dpart, c->d_ftmp, c->d_fcx, c->d_hf, c->d_gpart,
                  c->d_eigA[0], c->d_eigA[1], c->d_eigV, c->d_eigw, c->d_eigpart, c->d_bar, c->d_tbar,
                  c->d_eigres, c->d_eigrot, c->d_small[0], c->d_small[1], c->d_small[2],
                  c->d_small[3], c->d_small[4], c->d_small[5], c->d_gate,
                  c->d_stats, c->d_tcA[0], c->d_tcA[1], c->d_tcA[2], c->d_tcB[0],
                  c->d_tcB[1], c->d_tcB[2], c->d_tcRotA[0], c->d_tcRotA[1], c->d_tcRotA[2],
                  c->d_tcPart, c->d_netpart, c->d_trid, c->d_ozA, c->d_ozB, c->d_ozE,
                  c->d_ozP, c->d_trivec, c->d_ozgA, c->d_ozgB, c->d_ozgP, c->d_ozgE, c->d_dop[0], c->d_dop[1], c->d_dop[2],
                  c->d_dope[0], c->d_dope[1], c->d_dope[2],
                  c->d_dft[0][0], c->d_dft[0][1], c->d_dft[1][0], c->d_dft[1][1],
                  c->d_dft[2][0], c->d_dft[2][1], c->d_dfte[0][0], c->d_dfte[0][1],
                  c->d_dfte[1][0], c->d_dfte[1][1], c->d_dfte[2][0], c->d_dfte[2][1]};
  for (void* p : ptrs)
    if (p) cudaFree(p);
}

// BF16 operand pieces (up to `pieces`) and the FP32 split-K partials of the
// tensor-core forms; pieces already present are kept.
static sky_status alloc_tc_scratch(Ctx* c, int pieces) {
  const int Imax = c->max_states > 0 ? c->max_states : 1;
  const long long V = 2LL * c->G;
  size_t pa, pb, pra, part;
  tc_scratch_sizes(Imax, V, c->num_sms, &pa, &pb, &pra, &part);
  sky_status s = SKY_OK;
  for (int k = 0; k < pieces && s == SKY_OK; ++k) {
    if (c->d_tcA[k]) continue;
    unsigned short *x = nullptr, *y = nullptr, *z = nullptr;
    s = dalloc(c, &x, pa);
    if (s == SKY_OK) s = dalloc(c, &y, pb);
    if (s == SKY_OK) s = dalloc(c, &z, pra);
    if (s != SKY_OK) {
      if (x) cudaFree(x);
      if (y) cudaFree(y);
      if (z) cudaFree(z);
      return s;
    }
    c->d_tcA[k] = x; c->d_tcB[k] = y; c->d_tcRotA[k] = z;
  }
  if (s == SKY_OK && !c->d_tcPart) {
    float* p = nullptr;
    s = dalloc(c, &p, part);
    c->d_tcPart = p;
    c->tc_partial_elems = part;
  }
  return s;
}

// Digit buffers, exponents and partials of the tensor-core
// split GEMMs: the overlap and recombination of the FP64 and FP32 forms
// (when oz_on) and the eigensolver's I x I products (from kOzZgemmMin
// states on, every form).  Buffers already present and large enough are kept;
// smaller ones are replaced (callers synchronise the stream first).
static sky_status alloc_oz_scratch(Ctx* c, bool overlap_too) {
  const int Imax = c->max_states > 0 ? c->max_states : 1;
  size_t ae, be, ee, pe;
  oz_scratch_sizes(overlap_too ? c->prec : SKY_F64, overlap_too ? Imax : 0, overlap_too ? 2LL * c->G : 0,
                   c->num_sms, &ae, &be, &ee, &pe);
  if (Imax >= kOzZgemmMin) {   // the I x I products: 2 I rows of ld = round_up(2 I, 8)
    const size_t zb = (size_t)6 * 2 * Imax * (size_t)((2 * Imax + 7) / 8 * 8);
    if (zb > be) be = zb;
    if (zb / 2 > ae) ae = zb / 2;
    if ((size_t)2 * Imax * Imax > pe) pe = (size_t)2 * Imax * Imax;
  }
  if (ee < (size_t)(2 * Imax + 2LL * c->G + 64)) ee = (size_t)(2 * Imax + 2LL * c->G + 64);
  if (c->d_ozB && c->oz_a_elems >= ae && c->oz_b_elems >= be && c->oz_p_elems >= pe)
    return SKY_OK;
  unsigned short *A = nullptr, *Bp = nullptr;
  int* E = nullptr;
  float2* P = nullptr;
  sky_status s = dalloc(c, &A, ae);
  if (s == SKY_OK) s = dalloc(c, &Bp, be);
  if (s == SKY_OK) s = dalloc(c, &E, ee);
  if (s == SKY_OK) s = dalloc(c, &P, pe);
  if (s != SKY_OK) {
    void* ptrs[] = {A, Bp, E, P};
    for (void* p : ptrs)
      if (p) cudaFree(p);
    return s;
  }
  void* old[] = {c->d_ozA, c->d_ozB, c->d_ozE, c->d_ozP};
  for (void* p : old)
    if (p) cudaFree(p);
  c->d_ozA = A; c->d_ozB = Bp; c->d_ozE = E; c->d_ozP = P;
  c->oz_a_elems = ae; c->oz_b_elems = be; c->oz_p_elems = pe;
  return SKY_OK;
}

static size_t scratch_budget() {
  const char* s = getenv("SKY_SCRATCH_MB");
  if (s && atol(s) > 0) return (size_t)atol(s) << 20;
  return (size_t)2048 << 20;
}

static std::atomic<unsigned long long> g_launches{0};
void note_launch(unsigned n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

}  // namespace sky

using namespace sky;

extern "C" {

int sky_supported_size(int n, sky_prec prec) { return size_ok(n, prec) ? 1 : 0; }

unsigned long long sky_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

int sky_tri_team_plan(int np, const int* n, int blocks, int* team, int* first, int* count) {
  return tri_team_plan(np, n, blocks, team, first, count);
}

sky_status sky_init(sky_ctx** out, const int grid[3], const double dx[3], const sky_skyrme* params,
                    const double twist[3], sky_prec prec, int max_states, void* stream) {
  if (!out) return SKY_EINVAL;
  *out = nullptr;
  if (!grid || !dx || !params || max_states < 0) return SKY_EINVAL;
  if (prec != SKY_F64 && prec != SKY_F32 && prec != SKY_F32_BF16X3 && prec != SKY_F32_BF16X6)
    return SKY_EUNSUPPORTED;
  for (int j = 0; j < 3; ++j) {
    if (!size_ok(grid[j], prec)) return SKY_EUNSUPPORTED;
    if (!(dx[j] > 0.0)) return SKY_EINVAL;
  }
  sky_ctx* c = new (std::nothrow) sky_ctx();
  if (!c) return SKY_ENOMEM;
  std::memset(static_cast<Ctx*>(c), 0, sizeof(Ctx));
  c->stream = (cudaStream_t)stream;
  c->prec = prec;
  c->max_states = max_states;
  c->csize = prec == SKY_F64 ? 16 : 8;
  c->G = 1;
  for (int j = 0; j < 3; ++j) {
    c->n[j] = grid[j];
    c->dx[j] = dx[j];
    c->L[j] = grid[j] * dx[j];
    c->theta[j] = twist ? twist[j] : 0.0;
    c->G *= grid[j];
  }
  c->dV = dx[0] * dx[1] * dx[2];
  c->cp = couplings(*params);
  c->damp_E0[0] = c->damp_E0[1] = NAN;
  cudaError_t e = cudaGetDevice(&c->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
  if (e != cudaSuccess) {
    cudaGetLastError();
    delete c;
    return SKY_ECUDA;
  }
  const long long G = c->G, V = 2 * G;
  const int Imax = max_states > 0 ? max_states : 1;
  const int m = Imax + (Imax & 1);
  size_t per_state = (size_t)3 * V * c->csize;
  size_t chunk = scratch_budget() / per_state;
  if (chunk < 1) chunk = 1;
  if (chunk > (size_t)Imax) chunk = Imax;
  c->chunk = (int)chunk;
  c->red_nblk = (int)((2 * G + 4095) / 4096);
  if (c->red_nblk < 1) c->red_nblk = 1;
  if (c->red_nblk > 64) c->red_nblk = 64;
  c->ov_slots = overlap_slots(c->num_sms);
  c->line_yz = 128;
  c->line_x = 64;
  c->ov_waves = 1;
  c->tc_waves = 2;
  c->wait_spins = kBarrierSpins;
  c->jac_max_sweeps = kJacMaxSweeps;
  c->eig_method = SKY_EIG_AUTO;
  c->line_arith = prec == SKY_F64 ? 1 : 0;   // the tensor-core operator once built
  size_t gpart = 0;
  for (int I = 1; I <= Imax; ++I) {   // room for the largest tunable split count
    const size_t need = overlap_partial_elems(I, V, kMaxOverlapWaves * c->ov_slots);
    if (need > gpart) gpart = need;
  }
  c->gpart_elems = gpart;

  sky_status s = SKY_OK;
#define ALLOC(ptr, n) if (s == SKY_OK) s = dalloc(c, &(ptr), (size_t)(n))
  ALLOC(c->d_status, 1);
  for (int j = 0; j < 3; ++j) {
    ALLOC(c->d_kt[j], grid[j]);
    ALLOC(c->d_ktdd[j], grid[j]);
    ALLOC(c->d_ktf[j], grid[j]);
    ALLOC(c->d_kp[j], grid[j]);
  }
  ALLOC(c->d_damp[0], G);
  ALLOC(c->d_damp[1], G);
  ALLOC(c->d_coul, G);
  if (s == SKY_OK) {
    void* p = nullptr;
    e = cudaMalloc(&p, chunk * per_state);
    if (e == cudaSuccess && fill_nan()) e = cudaMemset(p, 0xFF, chunk * per_state);
    if (e != cudaSuccess) { cudaGetLastError(); s = set_err(c, SKY_ENOMEM, "scratch allocation failed"); }
    c->d_gscr = p;
  }
  {
    // per-state reduction partials of h psi: the general path's blocks or the
    // fused FP32 path's (one per 32 lines along z at most)
    const long long fz = ((long long)grid[0] * grid[1] + 31) / 32;
    const long long nb = fz > c->red_nblk ? fz : c->red_nblk;
    ALLOC(c->d_red, (size_t)Imax * nb * 2);
  }
  if (prec != SKY_F64) {
    // fused h psi by default up to axis length 24 (measured faster there on
    // GB300: 16^3 1.6x, 24^3 1.3x); at 32 its per-line state limits the warps
    // per SM and the general passes are faster (the knob still selects it)
    ALLOC(c->d_hf, (size_t)5 * G);
    c->fused_h = grid[0] <= 24 && grid[1] <= 24 && grid[2] <= 24 ? 1 : 0;
  }
  ALLOC(c->d_dpart, (size_t)kDensSplits * 5 * G);
  ALLOC(c->d_ftmp, (size_t)16 * G);
  ALLOC(c->d_fcx, G);
  ALLOC(c->d_gpart, gpart);
  // eigensolver and small-matrix workspace: eig_batch problems of size Imax
  c->eig_batch = 2;
  c->eig_slot = (size_t)m * m;
  c->eig_slot_rot = (size_t)(m / 2 + 1);
  c->small_slot = (size_t)Imax * Imax;
  ALLOC(c->d_eigA[0], c->eig_slot * c->eig_batch);
  ALLOC(c->d_eigA[1], c->eig_slot * c->eig_batch);
  ALLOC(c->d_eigV, c->eig_slot * c->eig_batch);
  ALLOC(c->d_eigw, (2 * c->eig_slot_rot + 2) * c->eig_batch);
  ALLOC(c->d_bar, 2);
  ALLOC(c->d_tbar, (size_t)32 * kMaxBatch);
  ALLOC(c->d_eigres, kMaxBatch);
  if (s == SKY_OK) {
    char* p = nullptr;
    s = dalloc(c, &p, jacobi_rot_bytes(m) * c->eig_batch);
    c->d_eigrot = p;
  }
  for (int k = 0; k < 6; ++k) ALLOC(c->d_small[k], c->small_slot * c->eig_batch);
  c->tri_m = m;
  c->tri_slot = tri_slot_doubles(m);
  ALLOC(c->d_trid, c->tri_slot * c->eig_batch);
  if (s == SKY_OK && tri_vec_elems(m, c->eig_batch, c->num_sms) > 0) {
    ALLOC(c->d_trivec, tri_vec_elems(m, c->eig_batch, c->num_sms));
    c->tri_vec_slots = c->eig_batch < 8 ? c->eig_batch : 8;
  }
  ALLOC(c->d_gate, 8 * kMaxBatch);
  if (s == SKY_OK && is_tc(prec)) s = alloc_tc_scratch(c, tc_nsplit(prec));
  c->oz_on = is_tc(prec) ? 0 : 1;
  if (s == SKY_OK && (c->oz_on || Imax >= kOzZgemmMin)) s = alloc_oz_scratch(c, c->oz_on != 0);
  ALLOC(c->d_stats, 8);
  ALLOC(c->d_netpart, net_partial_elems(c->G));
  if (s == SKY_OK) {
    c->eig_grid_max = jacobi_max_grid(c);
    c->eig_grid = c->eig_grid_max < c->num_sms ? c->eig_grid_max : c->num_sms;   // one per SM
    c->eig_grid_auto = true;
    ALLOC(c->d_eigpart, (size_t)2 * c->eig_grid_max * kMaxBatch);
  }
#undef ALLOC
  if (s == SKY_OK) {
    // wavenumbers in FFT order: index a -> m = a (a < (n+1)/2) or a - n
    for (int j = 0; j < 3 && s == SKY_OK; ++j) {
      const int n = grid[j];
      double* kt = new double[n];
      double* kp = new double[n];
      float* kf = new float[n];
      float2* kdd = new float2[n];
      for (int a = 0; a < n; ++a) {
        const int mm = (a < (n + 1) / 2) ? a : a - n;
        kp[a] = 2.0 * M_PI * mm / c->L[j];
        kt[a] = kp[a] + c->theta[j] / c->L[j];
        kf[a] = (float)kt[a];
        // (k + theta/L) / n as the nearest float pair, in long double
        const long double kl = (2.0L * 3.141592653589793238462643383279502884L * mm +
                                (long double)c->theta[j]) / ((long double)c->L[j] * n);
        const float h = (float)kl;
        kdd[a] = make_float2(h, (float)(kl - (long double)h));
      }
      e = cudaMemcpy(c->d_kt[j], kt, n * sizeof(double), cudaMemcpyHostToDevice);
      if (e == cudaSuccess) e = cudaMemcpy(c->d_ktdd[j], kdd, n * sizeof(float2), cudaMemcpyHostToDevice);
      if (e == cudaSuccess) e = cudaMemcpy(c->d_kp[j], kp, n * sizeof(double), cudaMemcpyHostToDevice);
      if (e == cudaSuccess) e = cudaMemcpy(c->d_ktf[j], kf, n * sizeof(float), cudaMemcpyHostToDevice);
      delete[] kt; delete[] kp; delete[] kf; delete[] kdd;
      s = cuda_check(c, e, "wavenumber upload");
    }
  }
  if (s == SKY_OK) s = cuda_check(c, cudaMemset(c->d_status, 0, sizeof(int)), "status reset");
  if (s == SKY_OK) s = cuda_check(c, cudaMemset(c->d_stats, 0, 8 * sizeof(long long)), "stats reset");
  if (s == SKY_OK) s = cuda_check(c, cudaMemset(c->d_bar, 0, 2 * sizeof(unsigned)), "barrier reset");
  if (s == SKY_OK) s = tri_init(c);
  if (s == SKY_OK) s = deriv_tc_init(c);
  if (s == SKY_OK && c->d_dop[0] && c->d_dop[1] && c->d_dop[2]) c->line_arith = 2;
  if (s == SKY_OK) s = upload_twiddles_hamiltonian(c);
  if (s == SKY_OK) s = upload_twiddles_fields(c);
  if (s == SKY_OK) s = build_coulomb_table(c);
  if (s == SKY_OK) s = cuda_check(c, cudaStreamSynchronize(c->stream), "init sync");
  if (s != SKY_OK) {
    free_all(c);
    delete c;
    return s;
  }
  *out = c;
  return SKY_OK;
}

sky_status sky_destroy(sky_ctx* c) {
  if (!c) return SKY_EINVAL;
  cudaStreamSynchronize(c->stream);
  free_all(c);
  delete c;
  return SKY_OK;
}

sky_status sky_set_stream(sky_ctx* c, void* stream) {
  if (!c) return SKY_EINVAL;
  c->stream = (cudaStream_t)stream;
  return SKY_OK;
}

sky_status sky_sync(sky_ctx* c) {
  if (!c) return SKY_EINVAL;
  int st = 0;
  cudaError_t e = cudaMemcpyAsync(&st, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_check(c, e, "sync");
  if (st) {
    cudaMemsetAsync(c->d_status, 0, sizeof(int), c->stream);
    cudaStreamSynchronize(c->stream);
    const sky_status order[] = {SKY_ETIMEOUT, SKY_ENOTPD, SKY_ENOCONV, SKY_ENAN};
    for (sky_status k : order)
      if (st & SKY_STATUS_BIT(k))
        return set_err(c, k, "device status word 0x%x", st);
  }
  return SKY_OK;
}

const char* sky_last_error(const sky_ctx* c) { return c ? c->err : "null context"; }

sky_status sky_memcpy_h2d(sky_ctx* c, void* dst, const void* src, size_t bytes) {
  if (!c) return SKY_EINVAL;
  if (bytes == 0) return SKY_OK;
  if (!dst || !src) return set_err(c, SKY_EINVAL, "memcpy_h2d: null pointer");
  return cuda_check(c, cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, c->stream),
                    "memcpy_h2d");
}

sky_status sky_memcpy_d2h(sky_ctx* c, void* dst, const void* src, size_t bytes) {
  if (!c) return SKY_EINVAL;
  if (bytes == 0) return SKY_OK;
  if (!dst || !src) return set_err(c, SKY_EINVAL, "memcpy_d2h: null pointer");
  return cuda_check(c, cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, c->stream),
                    "memcpy_d2h");
}

sky_status sky_stats(sky_ctx* c, long long out[8], int reset) {
  if (!c || !out) return SKY_EINVAL;
  cudaError_t e = cudaMemcpyAsync(out, c->d_stats, 8 * sizeof(long long), cudaMemcpyDeviceToHost,
                                  c->stream);
  if (e == cudaSuccess && reset) e = cudaMemsetAsync(c->d_stats, 0, 8 * sizeof(long long), c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  return cuda_check(c, e, "stats");
}

#define CHECK_CTX()                                     \
  if (!c) return SKY_EINVAL;                            \
  if (I < 0 || I > c->max_states)                       \
    return set_err(c, SKY_EINVAL, "I=%d outside [0, %d]", I, c->max_states)

sky_status sky_apply_h(sky_ctx* c, const double* U, const double* B, const double* W,
                       const void* psi, void* hpsi, int I, double* eps, double* hnorm2) {
  CHECK_CTX();
  if (I == 0) return SKY_OK;
  if (!U || !B || !W || !psi || !hpsi) return set_err(c, SKY_EINVAL, "apply_h: null pointer");
  if (psi == hpsi) return set_err(c, SKY_EINVAL, "apply_h: psi and hpsi must differ");
  return apply_h_impl(c, U, B, W, psi, hpsi, I, eps, hnorm2);
}

sky_status sky_td_taylor(sky_ctx* c, const double* U, const double* B, const double* W,
                         const void* psi, void* out, void* work, int I, double tau, int order) {
  CHECK_CTX();
  if (I == 0) return SKY_OK;
  if (!U || !B || !W || !psi || !out || (order > 0 && !work))
    return set_err(c, SKY_EINVAL, "td_taylor: null pointer");
  if (order < 0 || order > 32) return set_err(c, SKY_EINVAL, "td_taylor: order %d outside [0, 32]", order);
  if (out == psi || work == psi || work == out)
    return set_err(c, SKY_EINVAL, "td_taylor: psi, out and work must be separate buffers");
  if (!(tau == tau) || tau > 1e300 || tau < -1e300) return set_err(c, SKY_EINVAL, "td_taylor: bad tau");
  return td_taylor_impl(c, U, B, W, psi, out, work, I, tau, order);
}

sky_status sky_derivative(sky_ctx* c, int axis, const void* src, void* dst, int n) {
  if (!c) return SKY_EINVAL;
  if (axis < 0 || axis > 2 || n < 0) return set_err(c, SKY_EINVAL, "derivative: axis %d, n %d", axis, n);
  if (n == 0) return SKY_OK;
  if (!src || !dst) return set_err(c, SKY_EINVAL, "derivative: null pointer");
  return derivative_impl(c, axis, src, dst, n);
}

sky_status sky_damped_step(sky_ctx* c, int q, const void* psi, const void* hpsi, const double* eps,
                           void* phi, int I, double x0, double E0, const float* w) {
  CHECK_CTX();
  if (I == 0) return SKY_OK;
  if (q != 0 && q != 1) return set_err(c, SKY_EINVAL, "damped_step: q must be 0 or 1");
  if (!psi || !hpsi || !eps || !phi) return set_err(c, SKY_EINVAL, "damped_step: null pointer");
  if (phi == psi || phi == hpsi) return set_err(c, SKY_EINVAL, "damped_step: phi must be a separate buffer");
  return damped_step_impl(c, q, psi, hpsi, eps, phi, I, x0, E0, w);
}

sky_status sky_overlap(sky_ctx* c, const void* a, const void* b, int I, double* X) {
  CHECK_CTX();
  if (I == 0) return SKY_OK;
  if (!a || !b || !X) return set_err(c, SKY_EINVAL, "overlap: null pointer");
  return overlap_impl(c, a, b, I, (double2*)X);
}

sky_status sky_orthonormalize(sky_ctx* c, const double* S, int I, double* C) {
  CHECK_CTX();
  if (I == 0) return SKY_OK;
  if (!S || !C || S == C) return set_err(c, SKY_EINVAL, "orthonormalize: bad pointers");
  return lowdin_impl(c, (const double2*)S, I, (double2*)C);
}

sky_status sky_subspace_diag(sky_ctx* c, const double* H, const double* C, int I, double* M,
                             double* eps) {
  CHECK_CTX();
  if (I == 0) return SKY_OK;
  if (!H || !C || !M || !eps) return set_err(c, SKY_EINVAL, "subspace_diag: null pointer");
  return subspace_impl(c, (const double2*)H, (const double2*)C, I, (double2*)M, eps);
}

static sky_status check_batch(sky_ctx* c, int nb, const int* I) {
  if (nb < 1 || nb > c->eig_batch || !I)
    return set_err(c, SKY_EINVAL, "batch of %d outside [1, %d]", nb, c->eig_batch);
  for (int b = 0; b < nb; ++b)
    if (I[b] < 1 || I[b] > c->max_states)
      return set_err(c, SKY_EINVAL, "I=%d outside [1, %d]", I[b], c->max_states);
  return SKY_OK;
}

sky_status sky_orthonormalize_batched(sky_ctx* c, int nb, const double* const* S, const int* I,
                                      double* const* C) {
  if (!c) return SKY_EINVAL;
  sky_status st = check_batch(c, nb, I);
  if (st != SKY_OK) return st;
  if (!S || !C) return set_err(c, SKY_EINVAL, "orthonormalize_batched: null pointer");
  for (int b = 0; b < nb; ++b)
    if (!S[b] || !C[b] || S[b] == C[b]) return set_err(c, SKY_EINVAL, "orthonormalize_batched: bad pointers");
  return lowdin_batch(c, nb, reinterpret_cast<const double2* const*>(S), I,
                      reinterpret_cast<double2* const*>(C));
}

sky_status sky_subspace_diag_batched(sky_ctx* c, int nb, const double* const* H,
                                     const double* const* C, const int* I, double* const* M,
                                     double* const* eps) {
  if (!c) return SKY_EINVAL;
  sky_status st = check_batch(c, nb, I);
  if (st != SKY_OK) return st;
  if (!H || !C || !M || !eps) return set_err(c, SKY_EINVAL, "subspace_diag_batched: null pointer");
  for (int b = 0; b < nb; ++b)
    if (!H[b] || !C[b] || !M[b] || !eps[b]) return set_err(c, SKY_EINVAL, "subspace_diag_batched: null pointer");
  return subspace_batch(c, nb, reinterpret_cast<const double2* const*>(H),
                        reinterpret_cast<const double2* const*>(C), I,
                        reinterpret_cast<double2* const*>(M), eps);
}

sky_status sky_subspace_diag_literal_batched(sky_ctx* c, int nb, const double* const* H,
                                             const double* const* C, const int* I,
                                             double* const* M, double* const* eps) {
  if (!c) return SKY_EINVAL;
  sky_status st = check_batch(c, nb, I);
  if (st != SKY_OK) return st;
  if (!H || !C || !M || !eps) return set_err(c, SKY_EINVAL, "subspace_diag_literal: null pointer");
  for (int b = 0; b < nb; ++b)
    if (!H[b] || !C[b] || !M[b] || !eps[b]) return set_err(c, SKY_EINVAL, "subspace_diag_literal: null pointer");
  return subspace_literal_batch(c, nb, reinterpret_cast<const double2* const*>(H),
                                reinterpret_cast<const double2* const*>(C), I,
                                reinterpret_cast<double2* const*>(M), eps);
}

sky_status sky_rotate(sky_ctx* c, const void* phi, const double* M, int I, void* psi_out) {
  CHECK_CTX();
  if (I == 0) return SKY_OK;
  if (!phi || !M || !psi_out) return set_err(c, SKY_EINVAL, "rotate: null pointer");
  if (phi == psi_out) return set_err(c, SKY_EINVAL, "rotate: output must not alias phi");
  return rotate_impl(c, phi, (const double2*)M, I, psi_out);
}

sky_status sky_densities(sky_ctx* c, const void* psi, int I, double* rho, double* tau, double* J,
                         double* divJ) {
  CHECK_CTX();
  if ((!psi && I > 0) || !rho || !tau || !divJ) return set_err(c, SKY_EINVAL, "densities: null pointer");
  return densities_impl(c, psi, I, rho, tau, J, divJ);
}

sky_status sky_mean_fields(sky_ctx* c, const double* rho, const double* tau, const double* divJ,
                           double* U, double* B, double* W) {
  if (!c) return SKY_EINVAL;
  if (!rho || !tau || !divJ || !U || !B || !W) return set_err(c, SKY_EINVAL, "mean_fields: null pointer");
  return mean_fields_impl(c, rho, tau, divJ, U, B, W);
}

sky_status sky_energy(sky_ctx* c, const double* rho, const double* tau, const double* divJ,
                      double* out) {
  if (!c) return SKY_EINVAL;
  if (!rho || !tau || !divJ || !out) return set_err(c, SKY_EINVAL, "energy: null pointer");
  return energy_impl(c, rho, tau, divJ, out);
}

sky_status sky_sp_spread(sky_ctx* c, const double* eps, const double* hnorm2, int A, double* out) {
  if (!c) return SKY_EINVAL;
  if (A < 0 || (A > 0 && (!eps || !hnorm2)) || !out) return set_err(c, SKY_EINVAL, "sp_spread: bad arguments");
  return sp_spread_impl(c, eps, hnorm2, A, out);
}

sky_status sky_set_prec(sky_ctx* c, sky_prec prec) {
  if (!c) return SKY_EINVAL;
  if (prec == c->prec) return SKY_OK;
  if (prec != SKY_F32 && !is_tc(prec)) return set_err(c, SKY_EINVAL, "unknown precision form %d", (int)prec);
  if (c->prec == SKY_F64)
    return set_err(c, SKY_EUNSUPPORTED, "an FP64 context keeps FP64 spinors; create an FP32 one");
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_check(c, e, "set_prec sync");
  const sky_prec old = c->prec;
  c->prec = prec;   // the scratch sizes depend on the form
  const sky_status s = is_tc(prec) ? alloc_tc_scratch(c, tc_nsplit(prec)) : alloc_oz_scratch(c, true);
  if (s != SKY_OK) {
    c->prec = old;
    return s;
  }
  if (!is_tc(prec)) c->oz_on = 1;
  return SKY_OK;
}

sky_status sky_tune_set(sky_ctx* c, sky_knob knob, int value) {
  if (!c) return SKY_EINVAL;
  switch (knob) {
    case SKY_KNOB_LINE_YZ:
      if (value != 32 && value != 64 && value != 128) break;
      c->line_yz = value;
      return SKY_OK;
    case SKY_KNOB_LINE_X:
      if (value != 16 && value != 32 && value != 64) break;
      c->line_x = value;
      return SKY_OK;
    case SKY_KNOB_OVERLAP_WAVES:
      if (value < 1 || value > kMaxOverlapWaves) break;
      c->ov_waves = value;
      return SKY_OK;
    case SKY_KNOB_TC_WAVES:
      if (value != 0 && value != 1 && value != 2 && value != 4) break;
      c->tc_waves = value;
      return SKY_OK;
    case SKY_KNOB_TC_TILE_N:
      if (value != 0 && value != 128 && value != 256) break;
      c->tc_tile_n = value;
      return SKY_OK;
    case SKY_KNOB_FUSED_H:
      if (value != 0 && value != 1) break;
      if (value == 1 && !fused_h_ok(c)) break;
      c->fused_h = value;
      return SKY_OK;
    case SKY_KNOB_JACOBI_BLOCKS:
      if (value < 1 || value > c->eig_grid_max) break;
      c->eig_grid = value;
      c->eig_grid_auto = false;
      return SKY_OK;
    case SKY_KNOB_WAIT_SPINS:
      if (value < 0) break;
      c->wait_spins = value == 0 ? 0 : (long long)value * 1000;
      return SKY_OK;
    case SKY_KNOB_JACOBI_MAX_SWEEPS:
      if (value < 1 || value > 1000) break;
      c->jac_max_sweeps = value;
      return SKY_OK;
    case SKY_KNOB_EIGEN_METHOD:
      if (value != SKY_EIG_AUTO && value != SKY_EIG_JACOBI && value != SKY_EIG_TRIDIAGONAL) break;
      c->eig_method = value;
      return SKY_OK;
    case SKY_KNOB_LINE_ARITH:
      if (value < 0 || value > 2) break;
      if (value >= 1 && c->prec != SKY_F64) break;
      if (value == 2 && !(c->d_dop[0] && c->d_dop[1] && c->d_dop[2])) break;
      c->line_arith = value;
      return SKY_OK;
    case SKY_KNOB_SPLIT_GEMM:
      if (value != 0 && value != 1) break;
      if (value == 1 && is_tc(c->prec)) break;
      if (value == 1) {
        cudaError_t e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) return cuda_check(c, e, "tune sync");
        const sky_status s = alloc_oz_scratch(c, true);
        if (s != SKY_OK) return s;
      }
      c->oz_on = value;
      return SKY_OK;
    default:
      return set_err(c, SKY_EINVAL, "unknown knob %d", (int)knob);
  }
  return set_err(c, SKY_EINVAL, "value %d not allowed for knob %d", value, (int)knob);
}

int sky_tune_get(const sky_ctx* c, sky_knob knob) {
  if (!c) return -1;
  switch (knob) {
    case SKY_KNOB_LINE_YZ: return c->line_yz;
    case SKY_KNOB_LINE_X: return c->line_x;
    case SKY_KNOB_OVERLAP_WAVES: return c->ov_waves;
    case SKY_KNOB_TC_WAVES: return c->tc_waves;
    case SKY_KNOB_TC_TILE_N: return c->tc_tile_n;
    case SKY_KNOB_FUSED_H: return c->fused_h && fused_h_ok(c) ? 1 : 0;
    case SKY_KNOB_JACOBI_BLOCKS: return c->eig_grid;
    case SKY_KNOB_JACOBI_BLOCKS_MAX: return c->eig_grid_max;
    case SKY_KNOB_WAIT_SPINS: return (int)(c->wait_spins / 1000);
    case SKY_KNOB_JACOBI_MAX_SWEEPS: return c->jac_max_sweeps;
    case SKY_KNOB_EIGEN_METHOD: return c->eig_method;
    case SKY_KNOB_SPLIT_GEMM: return c->oz_on;
    case SKY_KNOB_LINE_ARITH: return c->line_arith;
    default: return -1;
  }
}

sky_status sky_reserve_batch(sky_ctx* c, int nb) {
  if (!c) return SKY_EINVAL;
  if (nb < 1 || nb > kMaxBatch) return set_err(c, SKY_EINVAL, "batch of %d outside [1, %d]", nb, kMaxBatch);
  if (nb <= c->eig_batch) return SKY_OK;
  const int Imax = c->max_states > 0 ? c->max_states : 1;
  const int m = Imax + (Imax & 1);
  double2 *a0 = nullptr, *a1 = nullptr, *v = nullptr, *sm[6] = {nullptr};
  double* w = nullptr;
  char* rot = nullptr;
  sky_status s = dalloc(c, &a0, c->eig_slot * nb);
  if (s == SKY_OK) s = dalloc(c, &a1, c->eig_slot * nb);
  if (s == SKY_OK) s = dalloc(c, &v, c->eig_slot * nb);
  if (s == SKY_OK) s = dalloc(c, &w, (2 * c->eig_slot_rot + 2) * nb);
  if (s == SKY_OK) s = dalloc(c, &rot, jacobi_rot_bytes(m) * nb);
  for (int k = 0; k < 6 && s == SKY_OK; ++k) s = dalloc(c, &sm[k], c->small_slot * nb);
  double* trid = nullptr;
  double2* tvec = nullptr;
  if (s == SKY_OK) s = dalloc(c, &trid, c->tri_slot * nb);
  if (s == SKY_OK && tri_vec_elems(m, nb, c->num_sms) > 0)
    s = dalloc(c, &tvec, tri_vec_elems(m, nb, c->num_sms));
  if (s != SKY_OK) {
    void* ptrs[] = {a0, a1, v, w, rot, sm[0], sm[1], sm[2], sm[3], sm[4], sm[5], trid, tvec};
    for (void* p : ptrs)
      if (p) cudaFree(p);
    return s;
  }
  // grouped I x I products for batches of many problems: digits of every
  // problem's rows stacked (up to nb x Imax rows, capped at about 2 GiB)
  void *ga = nullptr, *gb = nullptr;
  float2* gp = nullptr;
  int* ge = nullptr;
  long long grows = 0, gld = 0;
  size_t gpe = 0;
  if (s == SKY_OK && nb > kOzGroupMin) {
    gld = (2LL * Imax + 7) / 8 * 8;
    const long long per_row = (long long)oz_group_slices() * 3 * gld * 2;   // A + B bytes
    const long long cap = 2LL << 30;
    grows = (long long)nb * Imax;
    if (grows * per_row > cap) grows = cap / per_row;
    gpe = (size_t)nb * 2 * (size_t)Imax * (size_t)Imax;
    if (gpe * sizeof(float2) > (size_t)cap) gpe = (size_t)cap / sizeof(float2);
    if (grows >= Imax) {
      unsigned short *pa = nullptr, *pb = nullptr;
      s = dalloc(c, &pa, (size_t)oz_group_slices() * grows * gld);
      if (s == SKY_OK) s = dalloc(c, &pb, (size_t)oz_group_slices() * 2 * grows * gld);
      if (s == SKY_OK) s = dalloc(c, &gp, gpe);
      if (s == SKY_OK) s = dalloc(c, &ge, (size_t)3 * grows);
      ga = pa;
      gb = pb;
      if (s != SKY_OK) {
        void* ptrs[] = {a0, a1, v, w, rot, sm[0], sm[1], sm[2], sm[3], sm[4], sm[5], trid, tvec,
                        ga, gb, gp, ge};
        for (void* p : ptrs)
          if (p) cudaFree(p);
        return s;
      }
    }
  }
  cudaStreamSynchronize(c->stream);   // no queued work may still use the old buffers
  void* old[] = {c->d_eigA[0], c->d_eigA[1], c->d_eigV, c->d_eigw, c->d_eigrot, c->d_small[0],
                 c->d_small[1], c->d_small[2], c->d_small[3], c->d_small[4], c->d_small[5],
                 c->d_trid, c->d_trivec};
  for (void* p : old)
    if (p) cudaFree(p);
  if (ga) {
    void* og[] = {c->d_ozgA, c->d_ozgB, c->d_ozgP, c->d_ozgE};
    for (void* p : og)
      if (p) cudaFree(p);
    c->d_ozgA = ga; c->d_ozgB = gb; c->d_ozgP = gp; c->d_ozgE = ge;
    c->ozg_rows = (int)grows; c->ozg_ld = gld; c->ozg_p_elems = gpe; c->ozg_np = nb;
  }
  c->d_trivec = tvec;
  c->tri_vec_slots = tvec ? (nb < 8 ? nb : 8) : 0;
  c->d_eigA[0] = a0; c->d_eigA[1] = a1; c->d_eigV = v; c->d_eigw = w; c->d_eigrot = rot;
  for (int k = 0; k < 6; ++k) c->d_small[k] = sm[k];
  c->d_trid = trid;
  c->eig_batch = nb;
  return SKY_OK;
}

sky_status sky_net_forward(sky_ctx* c, int q, const float* theta, const double* U,
                           const double* B, const double* W, double scale, float* ws, float* w) {
  if (!c) return SKY_EINVAL;
  if (q != 0 && q != 1) return set_err(c, SKY_EINVAL, "net_forward: q must be 0 or 1");
  if (!theta || !U || !B || !W || !ws || !w) return set_err(c, SKY_EINVAL, "net_forward: null pointer");
  if (!(scale >= 0.0 && scale <= 1.0)) return set_err(c, SKY_EINVAL, "net_forward: scale outside [0, 1]");
  return net_forward_impl(c, q, theta, U, B, W, scale, ws, w);
}

sky_status sky_net_backward(sky_ctx* c, const float* theta, float* ws, const double* abc,
                            const double* norm, double* grad, double* loss) {
  if (!c) return SKY_EINVAL;
  if (!theta || !ws || !abc || !norm || !grad || !loss)
    return set_err(c, SKY_EINVAL, "net_backward: null pointer");
  return net_backward_impl(c, theta, ws, abc, norm, grad, loss);
}

sky_status sky_net_adam(sky_ctx* c, float* theta, double* grad, double* m, double* v, int step,
                        double lr, double beta1, double beta2, double eps) {
  if (!c) return SKY_EINVAL;
  if (!theta || !grad || !m || !v) return set_err(c, SKY_EINVAL, "net_adam: null pointer");
  if (step < 1 || !(lr >= 0.0) || !(beta1 >= 0.0 && beta1 < 1.0) || !(beta2 >= 0.0 && beta2 < 1.0) ||
      !(eps >= 0.0))
    return set_err(c, SKY_EINVAL, "net_adam: bad hyper-parameters");
  return net_adam_impl(c, theta, grad, m, v, step, lr, beta1, beta2, eps);
}

sky_status sky_cross_overlap(sky_ctx* c, const void* a, const void* b, int I, double* X) {
  CHECK_CTX();
  if (I == 0) return SKY_OK;
  if (!a || !b || !X) return set_err(c, SKY_EINVAL, "cross_overlap: null pointer");
  return cross_overlap_impl(c, a, b, I, (double2*)X);
}

sky_status sky_precond_stats(sky_ctx* c, const void* psi, const void* phi, const void* ppsi, int I,
                             double* abc, double* norm) {
  CHECK_CTX();
  if ((I > 0 && (!psi || !phi || !ppsi)) || !abc || !norm)
    return set_err(c, SKY_EINVAL, "precond_stats: null pointer");
  return precond_stats_impl(c, psi, phi, ppsi, I, abc, norm);
}

}  // extern "C"
