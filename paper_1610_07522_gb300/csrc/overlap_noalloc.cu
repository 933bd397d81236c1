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
// address), so the device address is looked up once per device with
// cudaGetSymbolAddress, with that device current, on the first call made
// on it; that first call should therefore happen before any stream capture.
// All calls share the array: calls whose work overlaps on the GPU (for
// example on two streams at once) race on it.  Each call writes every
// partial entry it later reads, so nothing has to be cleared between calls.
#include <mutex>

#include "overlap_kernels.cuh"

namespace sky {
namespace {

constexpr size_t kNoallocElems = (size_t)1 << 20;   // 16 MiB of double2
constexpr int kNoallocMaxI = 1024;                   // I * I <= kNoallocElems
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double2 g_noalloc_partial[kNoallocElems];

std::mutex g_setup_mutex;
double2* g_partial_ptr[kMaxDevices] = {};
int g_num_sms[kMaxDevices] = {};

// Device address of the scratch array and the SM count of the current device,
// looked up on the first call on that device.
cudaError_t device_setup(int dev, double2** ptr, int* sms) {
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_partial_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partial);
    if (e != cudaSuccess) return e;
    int n = 0;
    e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    g_partial_ptr[dev] = static_cast<double2*>(p);
    g_num_sms[dev] = n;
  }
  *ptr = g_partial_ptr[dev];
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
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) return SKY_ECUDA;
  double2* part = nullptr;
  int sms = 0;
  if (device_setup(dev, &part, &sms) != cudaSuccess) {
    cudaGetLastError();
    return SKY_ECUDA;
  }
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
  k_overlap_reduce<<<div_up((long long)I * I, 256), 256, 0, s>>>(part, nsplit_eff, I, dV,
                                                                (double2*)X);
  note_launch();
  return cudaGetLastError() == cudaSuccess ? SKY_OK : SKY_ECUDA;
}
