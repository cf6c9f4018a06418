// Allocation-free pair energy (exx_pair_energy_noalloc, declared in
// include/exx.h).
//
// Some callers cannot call cudaMalloc: host codes that hand the whole device
// memory to their own pool allocator at start-up and forbid any other
// allocation, and codes that must not take the implicit device-wide
// synchronisation and latency an allocation can bring inside their iteration
// loop.  This entry point serves them: it runs the energy-only path of one
// orbital pair (co-density + x/y transforms, z transforms with the kernel
// multiply and Parseval sum, block reduction) on scratch that lives in the
// file-scope device arrays below, and never allocates device memory.
//
// The arrays are sized for grids up to EXX_NOALLOC_MAX_N points per axis
// (about 29 MB in total: 14.3 MB of spectrum and 14.3 MB of kernel table at
// n = 96); every GPU that loads the library keeps them until the process
// exits.  In host code an array's name is only a host-side
// stand-in, so the device addresses are looked up once per device with
// cudaGetSymbolAddress and passed to the kernels as plain pointers.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <vector>

#include "exx.h"
#include "exx_ops.cuh"

namespace exx_host {
bool kernel_spectrum_octant(int n, double h, int kind, double omega, double* out);
}
namespace exx {
const Ops* find_ops(int prec, int n);
}

constexpr int kNoallocMaxN = EXX_NOALLOC_MAX_N;
constexpr size_t kSpecElems = (size_t)(kNoallocMaxN + 1) * kNoallocMaxN * 2 * kNoallocMaxN;
// kernel table (exx::kernel_table_bytes(n, n, 4, false) / 4 floats for n <= max;
// n <= 96 never uses the folded layout)
constexpr size_t kKernElems = (size_t)(kNoallocMaxN + 1) * 2 * kNoallocMaxN * 2 * kNoallocMaxN;
constexpr int kTwElems = 7 * kNoallocMaxN;  // exx::twiddle_count(n) for n <= max
constexpr int kEpartElems = (kNoallocMaxN + 1) * ((2 * kNoallocMaxN + 31) / 32);

// Shared scratch of every call on a device (contents persist between calls):
// the pair's spectrum (complex), the kernel table, the twiddles, the
// column-block energy partials and the pair slot.
static __device__ __align__(256) float2 g_noalloc_spec[kSpecElems];
static __device__ __align__(256) float g_noalloc_kern[kKernElems];
static __device__ __align__(256) float2 g_noalloc_tw[kTwElems];
static __device__ __align__(256) double g_noalloc_epart[kEpartElems];
static __device__ __align__(256) int4 g_noalloc_pair[1];
static __device__ int g_noalloc_err[2];  // [0] set by a device-side wait that ran out; [1] test hook

// the stated footprint (about 29 MB) cannot drift from the array sizes
constexpr size_t kNoallocBytes = kSpecElems * sizeof(float2) + kKernElems * sizeof(float) +
                                 kTwElems * sizeof(float2) + kEpartElems * sizeof(double) +
                                 sizeof(int4) + 2 * sizeof(int);
static_assert(kNoallocBytes > 28u * 1000 * 1000 && kNoallocBytes < 29u * 1000 * 1000,
              "static scratch of exx_pair_energy_noalloc: about 29 MB");

namespace {

constexpr int kMaxN = kNoallocMaxN;

// Per-device addresses of the arrays and the (n, h, kernel) whose spectrum and
// twiddles they currently hold, guarded by the device's own mutex.
struct DeviceScratch {
  std::mutex mu;
  bool ready = false;
  float2* spec = nullptr;
  float* kern = nullptr;
  float2* tw = nullptr;
  double* epart = nullptr;
  int4* pair = nullptr;
  int* err = nullptr;
  CUtensorMap gmap{};  // TMA descriptor of the kernel table (ops->stage_table)
  int n = 0;
  double h = 0.0;
  int kind = -1;
};
constexpr int kMaxDevices = 64;
DeviceScratch g_noalloc_dev[kMaxDevices];

__global__ void k_noalloc_set_pair(int i, int j) { g_noalloc_pair[0] = make_int4(i, j, 0, 0); }

// E = h^3 * (sum of the column-block partials), fixed-order warp reduction;
// NaN (and the flag cleared) when a device-side wait of this pair ran out
__global__ void k_noalloc_pair_total(const double* __restrict__ epart, int nper, double h3,
                                     int* __restrict__ err, double* __restrict__ E) {
  double s = 0.0;
  for (int t = threadIdx.x; t < nper; t += 32) s += epart[t];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (threadIdx.x == 0) {
    *E = *err ? __longlong_as_double(0x7ff8000000000000LL) : h3 * s;
    *err = 0;
  }
}

// One-time set-up on the current device: device addresses of the arrays.
exx_status_t lookup_addresses(DeviceScratch& d) {
  if (cudaGetSymbolAddress(reinterpret_cast<void**>(&d.spec), g_noalloc_spec) != cudaSuccess ||
      cudaGetSymbolAddress(reinterpret_cast<void**>(&d.kern), g_noalloc_kern) != cudaSuccess ||
      cudaGetSymbolAddress(reinterpret_cast<void**>(&d.tw), g_noalloc_tw) != cudaSuccess ||
      cudaGetSymbolAddress(reinterpret_cast<void**>(&d.epart), g_noalloc_epart) != cudaSuccess ||
      cudaGetSymbolAddress(reinterpret_cast<void**>(&d.pair), g_noalloc_pair) != cudaSuccess ||
      cudaGetSymbolAddress(reinterpret_cast<void**>(&d.err), g_noalloc_err) != cudaSuccess) {
    cudaGetLastError();
    return EXX_ERR_CUDA;
  }
  d.ready = true;
  return EXX_OK;
}

// Kernel table (exx::build_kernel_table, FP32) and twiddles for (n, h, kind),
// built on the host and copied into the arrays; synchronises the stream.
exx_status_t load_tables(DeviceScratch& d, const exx::Ops* ops, int n, double h, int kind,
                         cudaStream_t st) {
  const size_t m = (size_t)n + 1;
  std::vector<double> G(m * m * m);
  if (!exx_host::kernel_spectrum_octant(n, h, kind, 0.0, G.data())) return EXX_ERR_INVALID_ARG;
  const double L = 2.0 * n;
  const double scale = 1.0 / (L * L * L);
  std::vector<double> gx(m), gy(2 * (size_t)n), gz(2 * (size_t)n);
  ops->gains(gx.data(), gy.data(), gz.data());
  std::vector<unsigned char> Gt(exx::kernel_table_bytes(n, n, sizeof(float), ops->table_fold_y));
  exx::build_kernel_table<float>(n, n, ops->table_fold_y, G.data(), scale, gx.data(), gy.data(),
                                 gz.data(), Gt.data());
  std::vector<float2> tw(exx::twiddle_count(n));
  exx::build_twiddles(n, reinterpret_cast<float*>(tw.data()));
  cudaError_t e = cudaMemcpyAsync(d.kern, Gt.data(), Gt.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d.tw, tw.data(), tw.size() * sizeof(float2), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess && ops->stage_table && !exx::make_ktab_map(&d.gmap, d.kern, n, n))
    e = cudaErrorInvalidValue;
  if (e == cudaSuccess) e = ops->setup();
  if (e != cudaSuccess) {
    cudaGetLastError();
    d.kind = -1;
    return EXX_ERR_CUDA;
  }
  d.n = n;
  d.h = h;
  d.kind = kind;
  return EXX_OK;
}

}  // namespace

extern "C" exx_status_t exx_pair_energy_noalloc(int n, double h, int kernel, const float* psi,
                                                int norb, int i, int j, double* E_dev,
                                                void* cuda_stream) {
  if (psi == nullptr || E_dev == nullptr || norb < 1 || i < 0 || j < 0 || i >= norb ||
      j >= norb || n < 2 || !(h > 0.0) || !std::isfinite(h))
    return EXX_ERR_INVALID_ARG;
  if (kernel != EXX_KERNEL_SINC && kernel != EXX_KERNEL_HOCKNEY) return EXX_ERR_INVALID_ARG;
  if (n > kMaxN) return EXX_ERR_NOT_SUPPORTED;  // beyond the static scratch
  const exx::Ops* ops = exx::find_ops(EXX_FP32, n);
  if (ops == nullptr || !ops->supported) return EXX_ERR_NOT_SUPPORTED;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return EXX_ERR_CUDA;
  }
  // Under the device's lock: set-up, and a copy of everything the launches
  // below read, so that no field of the shared record is read after the lock
  // is released (another thread may reload the tables for other (n, h, kernel)
  // meanwhile; its GPU work is ordered with this call's only by the caller).
  // A reload synchronises the caller's stream while holding the lock, so
  // calls on the same device from other threads wait until that stream drains.
  DeviceScratch local_copy;
  {
    DeviceScratch* d = &g_noalloc_dev[dev];
    std::lock_guard<std::mutex> lock(d->mu);
    if (!d->ready) {
      const exx_status_t s = lookup_addresses(*d);
      if (s != EXX_OK) return s;
    }
    if (d->n != n || d->h != h || d->kind != kernel) {
      const exx_status_t s = load_tables(*d, ops, n, h, kernel, st);
      if (s != EXX_OK) return s;
    }
    local_copy.spec = d->spec;
    local_copy.kern = d->kern;
    local_copy.tw = d->tw;
    local_copy.epart = d->epart;
    local_copy.pair = d->pair;
    local_copy.err = d->err;
    local_copy.gmap = d->gmap;
  }
  const DeviceScratch& d = local_copy;
  // Every scratch element read below is first written by this call (the pair
  // slot, the n-sized part of the spectrum, the column-block partials), so
  // nothing needs clearing.
  const long long n3 = (long long)n * n * n;
  k_noalloc_set_pair<<<1, 1, 0, st>>>(i, j);
  ops->fwd_xy(psi, nullptr, d.pair, 1, d.spec, d.tw, n3, st);
  ops->zconv(d.spec, d.kern, d.tw, &d.gmap, d.epart, d.err, 1, true, st);
  k_noalloc_pair_total<<<1, 32, 0, st>>>(d.epart, (n + 1) * ops->nyb, h * h * h, d.err, E_dev);
  if (cudaGetLastError() != cudaSuccess) return EXX_ERR_CUDA;
  return EXX_OK;
}
