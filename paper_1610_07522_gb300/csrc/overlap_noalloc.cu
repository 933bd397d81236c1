// sky_overlap_noalloc: the overlap matrix without a context and without any
// device allocation.  For callers that are not allowed to allocate device
// memory themselves -- for example code embedded in a host application whose
// allocator owns the whole device-memory budget, or a long-running service
// that must not risk an allocation failure mid-run -- and so cannot create a
// context (sky_init allocates).
//
// The split-K partial sums live in one file-scope device array of fixed size
// (kNoallocElems complex doubles = 16 MiB).  Every GPU that loads the library
// holds this array until the process exits.  Host code cannot pass the
// array's name to a kernel (on the host it names a stand-in, not the device
// address), and the device address belongs to the CUDA context current at
// the call (a device reset or another context on the same device gives
// another address), so every call looks it up with cudaGetSymbolAddress in
// the current context.  The first call in a context loads the library's
// device code there and should therefore happen before any stream capture;
// later lookups are host-side table reads.  All calls share the array: calls
// whose work overlaps on the GPU (for example on two streams at once) race on
// it.  Each call writes every partial entry it later reads, so nothing has to
// be cleared between calls.
#include <mutex>

#include "overlap_kernels.cuh"

namespace sky {
namespace {

constexpr size_t kNoallocElems = (size_t)1 << 20;   // 16 MiB of double2
constexpr int kNoallocMaxI = 1024;                   // I * I <= kNoallocElems
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double2 g_noalloc_partial[kNoallocElems];

std::mutex g_sms_mutex;
int g_num_sms[kMaxDevices] = {};

// SM count of device dev (a device property: cached per device number).
cudaError_t device_sms(int dev, int* sms) {
  std::lock_guard<std::mutex> lock(g_sms_mutex);
  if (!g_num_sms[dev]) {
    int n = 0;
    const cudaError_t e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    g_num_sms[dev] = n;
  }
  *sms = g_num_sms[dev];
  return cudaSuccess;
}

}  // namespace
}  // namespace sky

using namespace sky;

extern "C" sky_status sky_overlap_noalloc(const void* a, const void* b, int I, long long V,
                                          double dV, sky_prec prec, double* X, void* stream) {
  if (I == 0) return SKY_OK;
  if (!a || !b || !X || I < 0 || V <= 0) return SKY_EINVAL;
  if (I > kNoallocMaxI) return SKY_EINVAL;   // the partial tile would not fit the scratch
  if (prec != SKY_F64 && prec != SKY_F32) return SKY_EUNSUPPORTED;
  // an error left pending by the caller's earlier work is not this call's:
  // leave it for the caller's own checks and do nothing
  if (cudaPeekAtLastError() != cudaSuccess) return SKY_ECUDA;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return SKY_ECUDA;
  int sms = 0;
  void* p = nullptr;
  if (device_sms(dev, &sms) != cudaSuccess || cudaGetSymbolAddress(&p, g_noalloc_partial) != cudaSuccess) {
    cudaGetLastError();   // the error just raised is this call's own
    return SKY_ECUDA;
  }
  double2* part = static_cast<double2*>(p);
  const int nt = (I + BM - 1) / BM;
  const int ntiles = nt * (nt + 1) / 2;
  const long long kblocks = (V + BK - 1) / BK;
  long long nsplit = (4LL * sms + ntiles - 1) / ntiles;
  const long long fit = (long long)(kNoallocElems / ((size_t)I * (size_t)I));
  if (nsplit > fit) nsplit = fit;
  if (nsplit > kblocks) nsplit = kblocks;
  if (nsplit < 1) nsplit = 1;
  const long long kchunk = ((kblocks + nsplit - 1) / nsplit) * BK;
  const int nsplit_eff = (int)((V + kchunk - 1) / kchunk);
  cudaStream_t s = (cudaStream_t)stream;
  dim3 grid(ntiles, nsplit_eff);
  if (prec == SKY_F64)
    k_overlap<double2><<<grid, 256, 0, s>>>((const double2*)a, (const double2*)b, I, V, kchunk, part);
  else
    k_overlap<float2><<<grid, 256, 0, s>>>((const float2*)a, (const float2*)b, I, V, kchunk, part);
  note_launch();
  if (cudaGetLastError() != cudaSuccess) return SKY_ECUDA;
  k_overlap_reduce<<<div_up((long long)I * I, 256), 256, 0, s>>>(part, nsplit_eff, I, dV,
                                                                (double2*)X);
  note_launch();
  return cudaGetLastError() == cudaSuccess ? SKY_OK : SKY_ECUDA;
}
