// Allocation-free fast-diagonalisation apply for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: code that runs while another component owns the device
// allocator (a framework with its own memory pool, a real-time loop with a fixed memory budget,
// a host that forbids allocation after start-up). This entry point needs no context and
// allocates nothing: the two intermediate tensors of the six mode products live in a file-scope
// static device array of fixed size, present on every GPU that loads the library until exit.
//
// The array's name in host code is only a host-side stand-in, not a device address. The first
// call on each device (made with that device current) obtains the device address with
// cudaGetSymbolAddress and caches it; make that first call before any stream capture.
// Every call shares the one array, so calls whose executions overlap on the GPU (different
// streams, or concurrent host threads) race on it; serialise them. Each mode product writes
// every element it later reads, so no part of the array has to start at zero.
#include <mutex>

#include "internal.h"
#include "stokes_hp.h"

namespace shp {
namespace {

constexpr int64_t kNoallocTensor = int64_t(1) << 19;   // entries per intermediate tensor
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_fd_scratch[2 * kNoallocTensor];

std::mutex g_mutex;
double* g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of g_fd_scratch on the current device (set up on first use).
cudaError_t scratch_address(double** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_fd_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

}  // namespace
}  // namespace shp

extern "C" int stokes_fd_apply_noalloc(int n1, int n2, int n3, const double* U1, const double* U2,
                                       const double* U3, const double* lam1, const double* lam2,
                                       const double* lam3, double scale, const double* x,
                                       double* y, void* stream) {
  using namespace shp;
  if (n1 < 1 || n2 < 1 || n3 < 1 || !U1 || !U2 || !U3 || !lam1 || !lam2 || !lam3 || !x || !y ||
      !(scale > 0.0))
    return STOKES_ERR_ARG;
  if ((int64_t)n1 * n2 * n3 > kNoallocTensor) return STOKES_ERR_ARG;
  // every one of the six mode products must fit the device's shared memory per block (staged
  // lines of the contracted extent); checked before anything is launched
  int dev = -1, smem_max = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) !=
          cudaSuccess)
    return STOKES_ERR_CUDA;
  double* scratch = nullptr;
  if (scratch_address(&scratch) != cudaSuccess) return STOKES_ERR_CUDA;
  double* f1 = scratch;
  double* f2 = scratch + kNoallocTensor;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const Dims d{n1, n2, n3};
  const double* U[3] = {U1, U2, U3};
  const int n[3] = {n1, n2, n3};
  auto job = [&](const double* X, double* Y, int k, int trans, bool last_forward) {
    ModeArgs<double> m{};
    m.X = X;
    m.Y = Y;
    m.U = U[k];
    m.ld = n[k];
    m.trans = trans;
    m.m = n[k];
    m.in = d;
    m.axis = k + 1;
    if (last_forward) {
      m.lam1 = lam1;
      m.lam2 = lam2;
      m.lam3 = lam3;
      m.scale = scale;
    }
    m.post = 1.0;
    return m;
  };
  const ModeArgs<double> seq[6] = {job(x, f1, 0, 1, false),  job(f1, f2, 1, 1, false),
                                   job(f2, f1, 2, 1, true),  job(f1, f2, 2, 0, false),
                                   job(f2, f1, 1, 0, false), job(f1, y, 0, 0, false)};
  for (const ModeArgs<double>& m : seq)
    if (mode_product_smem(m) > smem_max) return STOKES_ERR_ARG;
  // each launch's own status; the first failure stops the sequence
  for (const ModeArgs<double>& m : seq)
    if (mode_product<double>(m, s) != cudaSuccess) return STOKES_ERR_CUDA;
  return STOKES_OK;
}
