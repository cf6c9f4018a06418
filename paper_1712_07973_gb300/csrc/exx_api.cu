// C ABI of the exact-exchange operator (declared in include/exx.h).
//
// A plan holds the FP64-built kernel spectrum (Sec. 2.1.2 of arXiv
// 1712.07973: Green's function on the mesh, applied by a zero-padded FFT),
// the FFT twiddles, the pair-tile schedule over the N(N+1)/2 pairs (Sec. 2,
// pair-count paragraph; Table pscount) and the device workspace of one tile.
// exx_apply / exx_energy enqueue the tile pipeline behind the caller's stream:
//   fwd_xy -> zconv -> pair_energy [-> inv_yx -> accum]   per pair tile
//   exx_total [-> convert]                                once
// With two or three lanes the transforms of consecutive tiles run on the
// lanes' internal streams (forked from and joined back into the caller's
// stream through events); the accumulation stays on the caller's stream in
// tile order.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "exx.h"
#include "exx_ops.cuh"

namespace exx_host {
bool kernel_spectrum_octant(int n, double h, int kind, double omega, double* out);
}

namespace exx {

// ---------------------------------------------------------------- registry
#define EXX_SIZES(X)                                                                         \
  X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(12) X(14) X(16) X(18) X(20) X(24) X(28)    \
  X(32) X(36) X(40) X(48) X(56) X(64) X(72) X(80) X(96) X(112) X(128) X(160)

// periodic boundary conditions: half grids (grid = 2 N)
#define EXX_PSIZES(X) X(4) X(6) X(8) X(12) X(16) X(24) X(32) X(48) X(64) X(96)
// slab boundary conditions: half grids (grid = 2 N); wire: grids
#define EXX_SSIZES(X) X(4) X(8) X(16) X(24) X(32) X(48)
#define EXX_WSIZES(X) X(8) X(16) X(32) X(48) X(64) X(96)

#define EXX_DECL(N) const Ops* ops_f32_##N(); const Ops* ops_f64_##N();
EXX_SIZES(EXX_DECL)
#undef EXX_DECL
#define EXX_DECL(N) const Ops* ops_pf32_##N(); const Ops* ops_pf64_##N();
EXX_PSIZES(EXX_DECL)
#undef EXX_DECL
#define EXX_DECL(N) const Ops* ops_sf32_##N(); const Ops* ops_sf64_##N();
EXX_SSIZES(EXX_DECL)
#undef EXX_DECL
#define EXX_DECL(N) const Ops* ops_wf32_##N(); const Ops* ops_wf64_##N();
EXX_WSIZES(EXX_DECL)
#undef EXX_DECL

// slab grid n = 2 N
static const Ops* lookup_ops_slab(int prec, int n) {
  if (n % 2 != 0) return nullptr;
  switch (n / 2) {
#define EXX_CASE(N) \
  case N:           \
    return prec == EXX_FP64 ? ops_sf64_##N() : ops_sf32_##N();
    EXX_SSIZES(EXX_CASE)
#undef EXX_CASE
    default:
      return nullptr;
  }
}

static const Ops* lookup_ops_wire(int prec, int n) {
  switch (n) {
#define EXX_CASE(N) \
  case N:           \
    return prec == EXX_FP64 ? ops_wf64_##N() : ops_wf32_##N();
    EXX_WSIZES(EXX_CASE)
#undef EXX_CASE
    default:
      return nullptr;
  }
}

// periodic grid n = 2 N
static const Ops* lookup_ops_periodic(int prec, int n) {
  if (n % 2 != 0) return nullptr;
  switch (n / 2) {
#define EXX_CASE(N) \
  case N:           \
    return prec == EXX_FP64 ? ops_pf64_##N() : ops_pf32_##N();
    EXX_PSIZES(EXX_CASE)
#undef EXX_CASE
    default:
      return nullptr;
  }
}

static const Ops* lookup_ops(int prec, int n) {
  switch (n) {
#define EXX_CASE(N) \
  case N:           \
    return prec == EXX_FP64 ? ops_f64_##N() : ops_f32_##N();
    EXX_SIZES(EXX_CASE)
#undef EXX_CASE
    default:
      return nullptr;
  }
}

const Ops* find_ops(int prec, int n) { return lookup_ops(prec, n); }

// ------------------------------------------------------ pair enumeration
// Global pair id of (i, j), i <= j, in row-major order over the upper
// triangle: g(i, j) = i N - i (i - 1) / 2 + (j - i).
__host__ __device__ inline long long tri_start(long long i, long long N) {
  return i * N - (i * (i - 1)) / 2;
}
// Inverse of g: the row i is the largest with tri_start(i) <= g (closed-form
// estimate, then exact integer correction), j = g - tri_start(i) + i.
__host__ __device__ inline void tri_decode(long long g, long long N, int* pi, int* pj) {
  const double b = 2.0 * (double)N + 1.0;
  double disc = b * b - 8.0 * (double)g;
  if (disc < 0.0) disc = 0.0;
  long long i = (long long)((b - sqrt(disc)) * 0.5);
  if (i < 0) i = 0;
  if (i > N - 1) i = N - 1;
  while (i + 1 <= N - 1 && tri_start(i + 1, N) <= g) ++i;
  while (i > 0 && tri_start(i, N) > g) --i;
  *pi = (int)i;
  *pj = (int)(g - tri_start(i, N) + i);
}

// ------------------------------------------------- size-independent kernels
// Per-pair energy: E_ij = h^3 sum of the zconv block partials (one warp per
// pair, fixed reduction order).
__global__ void k_pair_energy(const double* __restrict__ epart, int nper,
                              const int4* __restrict__ pairs, int npair, double h3,
                              double* __restrict__ Epair) {
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= npair) return;
  double s = 0.0;
  for (int t = lane; t < nper; t += 32) s += epart[(long long)w * nper + t];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) Epair[pairs[w].z] = h3 * s;
}

// E_x = -(alpha/2) sum_{i,j} f_i f_j E_ij = -(alpha/2) sum_{i<=j} (2 - d_ij) f_i f_j E_ij
// (Eq. HF).  One block, fixed-order tree reduction; pairs decoded on device.
__global__ void k_exx_total(const double* __restrict__ Epair, long long P, int N,
                            const double* __restrict__ occ, double alpha, double* __restrict__ E) {
  __shared__ double red[256];
  double s = 0.0;
  for (long long g = threadIdx.x; g < P; g += blockDim.x) {
    int i, j;
    tri_decode(g, N, &i, &j);
    const double m = (i == j) ? 1.0 : 2.0;
    s += m * occ[i] * occ[j] * Epair[g];
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *E = -0.5 * alpha * red[0];
}

__global__ void k_to_float(const double* __restrict__ a, float* __restrict__ b, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}

struct Tile {
  int off, count;      // slice of the pair table
  int i0, ti, j0, tj;  // orbital blocks
  int diag;
};

// Tiles of blocks of T orbitals over the triangle bi <= bj, row-major.
static std::vector<Tile> make_tiles(int norb, int T) {
  std::vector<Tile> tiles;
  const int nb = (norb + T - 1) / T;
  int off = 0;
  for (int bi = 0; bi < nb; ++bi)
    for (int bj = bi; bj < nb; ++bj) {
      Tile t;
      t.i0 = bi * T;
      t.ti = std::min(T, norb - t.i0);
      t.j0 = bj * T;
      t.tj = std::min(T, norb - t.j0);
      t.diag = (bi == bj);
      t.off = off;
      t.count = t.diag ? t.ti * (t.ti + 1) / 2 : t.ti * t.tj;
      off += t.count;
      tiles.push_back(t);
    }
  return tiles;
}

// Largest-first onto the least-loaded rank (ties: lower tile index first,
// lowest rank): deterministic, imbalance at most one tile.
static std::vector<int> shard_owners(const std::vector<Tile>& tiles, int nranks) {
  std::vector<int> order(tiles.size());
  for (size_t k = 0; k < order.size(); ++k) order[k] = (int)k;
  std::stable_sort(order.begin(), order.end(),
                   [&](int a, int b) { return tiles[a].count > tiles[b].count; });
  std::vector<long long> load(nranks, 0);
  std::vector<int> owner(tiles.size(), 0);
  for (int k : order) {
    int r = 0;
    for (int q = 1; q < nranks; ++q)
      if (load[q] < load[r]) r = q;
    owner[k] = r;
    load[r] += tiles[k].count;
  }
  return owner;
}

}  // namespace exx

using namespace exx;

constexpr int kMaxLanes = 3;      // pipeline lanes a plan can hold
constexpr int kDefaultLanes = 2;  // two measured 4% faster than one at 96^3 (unclustered slabs)

struct exx_plan_s {
  int n = 0, N = 0, prec = 0, kind = 0;
  unsigned flags = 0;
  double h = 0.0, alpha = 0.0, omega = 0.0;
  std::vector<double> occ;
  const Ops* ops = nullptr;
  int T = 0;
  std::vector<Tile> tiles;
  std::vector<char> mine;  // tiles this plan processes (all unless sharded)
  bool sharded = false;
  int maxpairs = 0;
  long long P = 0;
  size_t ws = 0;
  int device = 0;
  std::string err;
  // device memory
  void* Gs = nullptr;
  void* tw = nullptr;
  void* twz = nullptr;  // twiddles of the z transform where its length differs
  double* d_occ = nullptr;
  int4* d_pairs = nullptr;
  double* epart = nullptr;
  double* Epair = nullptr;
  void* X2 = nullptr;
  void* V = nullptr;
  double* vacc = nullptr;
  double* E_dev = nullptr;
  int* d_err = nullptr;    // set by a device-side wait that ran out
  int fail_alloc = 0;      // test hook: this device allocation (1-based) reports out of memory
  int nalloc = 0;          // device allocations made by dalloc so far
  CUtensorMap gmap{};      // TMA descriptor of the kernel table (Ops::stage_table)
  void* h_psi = nullptr;  // exx_apply_host staging (allocated on first use)
  void* h_vx = nullptr;
  // pipeline lanes (run): lanes in use, lanes with workspaces, and the
  // workspaces, streams and events of lanes 1.. (lane 0 uses X2, V, epart)
  int lanes = 1, max_lanes = 1;
  void* X2x[kMaxLanes] = {};
  void* Vx[kMaxLanes] = {};
  double* epx[kMaxLanes] = {};
  cudaStream_t ls[kMaxLanes] = {};
  cudaEvent_t ev_fork = nullptr, ev_done[kMaxLanes] = {}, ev_free[kMaxLanes] = {};
  // exx_apply_host overlap: copy stream, per-orbital-block events
  cudaStream_t cst = nullptr;
  cudaEvent_t ev_start = nullptr, ev_join = nullptr;
  std::vector<cudaEvent_t> ev_in, ev_out;
  // per-kernel event timing (exx_profile_enable)
  bool prof = false;
  std::vector<cudaEvent_t> ev[EXX_NKINDS];  // start/stop pairs, in launch order
  size_t used[EXX_NKINDS] = {};
  double ms[EXX_NKINDS] = {};
  long long cnt[EXX_NKINDS] = {};
};

namespace {

const char* kStatus[] = {"EXX_OK", "EXX_ERR_INVALID_ARG", "EXX_ERR_CUDA", "EXX_ERR_OOM",
                         "EXX_ERR_TIMEOUT", "EXX_ERR_NOT_SUPPORTED"};

exx_status_t cuda_fail(exx_plan_t p, cudaError_t e) {
  if (p) p->err = cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? EXX_ERR_OOM : EXX_ERR_CUDA;
}

#define EXX_CUDA(p, call)                         \
  do {                                            \
    cudaError_t e_ = (call);                      \
    if (e_ != cudaSuccess) return cuda_fail(p, e_); \
  } while (0)

void free_plan(exx_plan_t p) {
  void* ptrs[] = {p->Gs,   p->tw,    p->twz,  p->d_occ, p->d_pairs, p->epart, p->Epair,
                  p->X2,   p->V,     p->vacc, p->E_dev, p->d_err,   p->h_psi, p->h_vx};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  for (int k = 0; k < EXX_NKINDS; ++k)
    for (cudaEvent_t e : p->ev[k]) cudaEventDestroy(e);
  for (cudaEvent_t e : p->ev_in) cudaEventDestroy(e);
  for (cudaEvent_t e : p->ev_out) cudaEventDestroy(e);
  if (p->ev_start) cudaEventDestroy(p->ev_start);
  if (p->ev_join) cudaEventDestroy(p->ev_join);
  if (p->cst) cudaStreamDestroy(p->cst);
  for (int l = 1; l < kMaxLanes; ++l)
    for (void* q : {p->X2x[l], p->Vx[l], static_cast<void*>(p->epx[l])})
      if (q) cudaFree(q);
  for (int l = 0; l < kMaxLanes; ++l) {
    if (p->ls[l]) cudaStreamDestroy(p->ls[l]);
    if (p->ev_done[l]) cudaEventDestroy(p->ev_done[l]);
    if (p->ev_free[l]) cudaEventDestroy(p->ev_free[l]);
  }
  if (p->ev_fork) cudaEventDestroy(p->ev_fork);
}

enum Kind { K_FWD = 0, K_ZCONV = 1, K_PAIRE = 2, K_INV = 3, K_ACCUM = 4, K_TOTAL = 5, K_CONV = 6 };

// Records a start/stop event pair on the launching stream around one launch.
struct ProfScope {
  exx_plan_t p;
  int kind;
  cudaStream_t st;
  cudaEvent_t stop = nullptr;
  ProfScope(exx_plan_t p_, int k, cudaStream_t s) : p(p_), kind(k), st(s) {
    if (!p->prof) return;
    std::vector<cudaEvent_t>& v = p->ev[kind];
    size_t& u = p->used[kind];
    while (v.size() < 2 * (u + 1)) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return;
      v.push_back(e);
    }
    cudaEventRecord(v[2 * u], st);
    stop = v[2 * u + 1];
    ++u;
  }
  ~ProfScope() {
    if (stop) cudaEventRecord(stop, st);
  }
};

template <typename T> exx_status_t dalloc(exx_plan_t p, T** out, size_t bytes) {
  if (p->fail_alloc > 0 && ++p->nalloc == p->fail_alloc) {
    p->err = "simulated allocation failure (EXX_TEST_FAIL_ALLOC)";
    return EXX_ERR_OOM;
  }
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, bytes ? bytes : 16);
  if (e != cudaSuccess) {
    cudaGetLastError();
    p->err = cudaGetErrorString(e);
    return EXX_ERR_OOM;
  }
  p->ws += bytes;
  *out = static_cast<T*>(q);
  return EXX_OK;
}

int default_tile(int N, int requested) {
  const char* env = std::getenv("EXX_TILE");
  int T = requested > 0 ? requested : (env ? std::atoi(env) : 8);
  if (T < 1) T = 1;
  if (T > 8) T = 8;
  return T < N ? T : N;
}

}  // namespace

// k_accum launch: vector width 2 when aligned, full-tile specialisations
template <typename R, int VEC>
void launch_accum_v(int mode, const R* psi, const R* V, double* acc, const double* occ,
                    const Tile& t, double c, double gs, long long n3, cudaStream_t st) {
  const int threads = 256;
  const unsigned blocks = (unsigned)((n3 / VEC + threads - 1) / threads);
  if (mode == 1)
    k_accum<R, 8, VEC, 1><<<blocks, threads, 0, st>>>(psi, V, acc, occ, t.i0, t.ti, t.j0, t.tj,
                                                       t.diag, c, gs, n3);
  else if (mode == 2)
    k_accum<R, 8, VEC, 2><<<blocks, threads, 0, st>>>(psi, V, acc, occ, t.i0, t.ti, t.j0, t.tj,
                                                       t.diag, c, gs, n3);
  else
    k_accum<R, 8, VEC, 0><<<blocks, threads, 0, st>>>(psi, V, acc, occ, t.i0, t.ti, t.j0, t.tj,
                                                       t.diag, c, gs, n3);
}
template <typename R>
void launch_accum(bool v2, int mode, const R* psi, const R* V, double* acc, const double* occ,
                  const Tile& t, double c, double gs, long long n3, cudaStream_t st) {
  if constexpr (sizeof(R) == 4) {  // four FP32 values per thread: -4% at 160^3
    if (v2 && (n3 % 4) == 0) {
      launch_accum_v<R, 4>(mode, psi, V, acc, occ, t, c, gs, n3, st);
      return;
    }
  }
  if (v2) launch_accum_v<R, 2>(mode, psi, V, acc, occ, t, c, gs, n3, st);
  else launch_accum_v<R, 1>(mode, psi, V, acc, occ, t, c, gs, n3, st);
}

extern "C" {

const char* exx_status_string(exx_status_t s) {
  return (s >= 0 && s <= EXX_ERR_NOT_SUPPORTED) ? kStatus[s] : "EXX_UNKNOWN_STATUS";
}

const char* exx_last_error(exx_plan_t p) { return p ? p->err.c_str() : ""; }

const char* exx_version(void) { return "exx-gb300 0.1 (sm_103a)"; }

exx_status_t exx_kernel_spectrum(int n, double h, int kernel, double omega, double* out_host) {
  if (n < 1 || !(h > 0.0) || out_host == nullptr) return EXX_ERR_INVALID_ARG;
  if (kernel < EXX_KERNEL_SINC || kernel > EXX_KERNEL_WIRE)
    return EXX_ERR_INVALID_ARG;
  return exx_host::kernel_spectrum_octant(n, h, kernel, omega, out_host) ? EXX_OK
                                                                          : EXX_ERR_INVALID_ARG;
}

static exx_status_t plan_create_impl(exx_plan_t* out, const int grid[3], const double h[3],
                                     double alpha, const double* occupations, int norb,
                                     int precision, int kernel, unsigned flags, double omega,
                                     void* cuda_stream);

exx_status_t exx_plan_create(exx_plan_t* out, const int grid[3], const double h[3], double alpha,
                             const double* occupations, int norb, int precision, int kernel,
                             unsigned flags, void* cuda_stream) {
  if (kernel == EXX_KERNEL_ERFC) return EXX_ERR_INVALID_ARG;  // needs omega: exx_plan_create_desc
  return plan_create_impl(out, grid, h, alpha, occupations, norb, precision, kernel, flags, 0.0,
                          cuda_stream);
}

exx_status_t exx_plan_create_desc(exx_plan_t* out, const exx_plan_desc* d, void* cuda_stream) {
  if (out == nullptr) return EXX_ERR_INVALID_ARG;
  *out = nullptr;
  if (d == nullptr) return EXX_ERR_INVALID_ARG;
  if (d->kernel == EXX_KERNEL_ERFC && !(d->omega > 0.0 && std::isfinite(d->omega)))
    return EXX_ERR_INVALID_ARG;
  return plan_create_impl(out, d->grid, d->h, d->alpha, d->occupations, d->norb, d->precision,
                          d->kernel, d->flags, d->kernel == EXX_KERNEL_ERFC ? d->omega : 0.0,
                          cuda_stream);
}

static exx_status_t plan_create_impl(exx_plan_t* out, const int grid[3], const double h[3],
                                     double alpha, const double* occupations, int norb,
                                     int precision, int kernel, unsigned flags, double omega,
                                     void* cuda_stream) {
  if (out == nullptr) return EXX_ERR_INVALID_ARG;
  *out = nullptr;
  if (grid == nullptr || h == nullptr || occupations == nullptr) return EXX_ERR_INVALID_ARG;
  if (norb < 1 || grid[0] < 2 || grid[1] < 2 || grid[2] < 2) return EXX_ERR_INVALID_ARG;
  if (!(h[0] > 0.0) || !(h[1] > 0.0) || !(h[2] > 0.0) || !std::isfinite(alpha))
    return EXX_ERR_INVALID_ARG;
  if (precision != EXX_FP64 && precision != EXX_FP32) return EXX_ERR_INVALID_ARG;
  if (kernel < EXX_KERNEL_SINC || kernel > EXX_KERNEL_WIRE)
    return EXX_ERR_INVALID_ARG;
  if (flags & ~((unsigned)EXX_FLAG_VX_FP64 | EXX_FLAG_TILE(15))) return EXX_ERR_INVALID_ARG;
  const int tile_req = (int)((flags >> 8) & 15u);
  if (tile_req > 8) return EXX_ERR_INVALID_ARG;
  for (int i = 0; i < norb; ++i)
    if (!std::isfinite(occupations[i])) return EXX_ERR_INVALID_ARG;
  if (grid[0] != grid[1] || grid[0] != grid[2] || h[0] != h[1] || h[0] != h[2])
    return EXX_ERR_NOT_SUPPORTED;
  const int n = grid[0];
  const Ops* ops = kernel == EXX_KERNEL_PERIODIC ? lookup_ops_periodic(precision, n)
                   : kernel == EXX_KERNEL_SLAB  ? lookup_ops_slab(precision, n)
                   : kernel == EXX_KERNEL_WIRE  ? lookup_ops_wire(precision, n)
                   : split_l1(2 * n) == 0       ? nullptr
                                                : lookup_ops(precision, n);
  if (ops == nullptr || !ops->supported) return EXX_ERR_NOT_SUPPORTED;
  // x and y transforms of length 2 nh, z transforms of length 2 nz: n (free
  // axis, padded) or n / 2 (periodic axis)
  const int nh = ops->n, nz = ops->nz;

  exx_plan_t p = new exx_plan_s();
  p->n = n;
  p->N = norb;
  p->prec = precision;
  p->kind = kernel;
  p->flags = flags;
  p->h = h[0];
  p->alpha = alpha;
  p->omega = omega;
  p->occ.assign(occupations, occupations + norb);
  p->ops = ops;
  p->P = (long long)norb * (norb + 1) / 2;
  cudaGetDevice(&p->device);
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);

  // pair tiles: blocks of T orbitals, tiles (bi, bj) with bi <= bj
  p->T = default_tile(norb, tile_req);
  const int T = p->T;
  std::vector<int4> pairs;
  for (Tile t : make_tiles(norb, T)) {
    t.off = (int)pairs.size();
    for (int a = 0; a < t.ti; ++a)
      for (int b = t.diag ? a : 0; b < t.tj; ++b) {
        const int i = t.i0 + a, j = t.j0 + b;
        pairs.push_back(make_int4(i, j, (int)tri_start(i, norb) + (j - i), 0));
      }
    t.count = (int)pairs.size() - t.off;
    p->maxpairs = std::max(p->maxpairs, t.count);
    p->tiles.push_back(t);
  }
  p->mine.assign(p->tiles.size(), 1);

  // kernel spectrum (FP64, host, one octant kz <= nz, kx, ky <= nh), scaled
  // by the inverse-FFT normalisation
  const size_t m = (size_t)nh + 1;
  std::vector<double> Gh(((size_t)nz + 1) * m * m);
  if (!exx_host::kernel_spectrum_octant(n, p->h, kernel, p->omega, Gh.data())) {
    delete p;
    return EXX_ERR_INVALID_ARG;
  }
  const double L = 2.0 * nh, LZ = 2.0 * nz;
  const double scale = 1.0 / (L * L * LZ);
  const size_t rs = precision == EXX_FP64 ? sizeof(double) : sizeof(float);
  const size_t cs = 2 * rs;
  // kernel table (scaled by 1/(L^2 LZ); for FP32 with the forward transforms'
  // gains divided out) and twiddle tables (exx_ops.cuh)
  std::vector<unsigned char> gbuf(exx::kernel_table_bytes(nh, nz, rs, ops->table_fold_y)),
      twbuf(exx::twiddle_count(nh) * cs), twzbuf(nz != nh ? exx::twiddle_count(nz) * cs : 0);
  std::vector<double> gx, gy, gz;
  if (ops->gains) {
    gx.resize(m);
    gy.resize(2 * (size_t)nh);
    gz.resize(2 * (size_t)nz);
    ops->gains(gx.data(), gy.data(), gz.data());
  }
  if (precision == EXX_FP64) {
    exx::build_kernel_table<double>(nh, nz, ops->table_fold_y, Gh.data(), scale, nullptr, nullptr,
                                    nullptr, gbuf.data());
    exx::build_twiddles(nh, reinterpret_cast<double*>(twbuf.data()));
    if (nz != nh) exx::build_twiddles(nz, reinterpret_cast<double*>(twzbuf.data()));
  } else {
    const bool g = !gx.empty();
    exx::build_kernel_table<float>(nh, nz, ops->table_fold_y, Gh.data(), scale,
                                   g ? gx.data() : nullptr, g ? gy.data() : nullptr,
                                   g ? gz.data() : nullptr, gbuf.data());
    exx::build_twiddles(nh, reinterpret_cast<float*>(twbuf.data()));
    if (nz != nh) exx::build_twiddles(nz, reinterpret_cast<float*>(twzbuf.data()));
  }

  const long long n3 = (long long)n * n * n;
  const size_t nper = m * (size_t)ops->nyb;
  exx_status_t st_;
  // test hook (EXX_TEST_FAIL_ALLOC=k, k >= 1): the plan's k-th device
  // allocation reports out of memory without calling cudaMalloc, so that the
  // clean-up of a failed creation is tested without exhausting the device
  {
    const char* hook = std::getenv("EXX_TEST_FAIL_ALLOC");
    if (hook != nullptr) p->fail_alloc = std::atoi(hook);
  }
#define EXX_ALLOC(ptr, bytes)                 \
  if ((st_ = dalloc(p, &(ptr), (bytes))) != EXX_OK) { \
    free_plan(p);                             \
    delete p;                                 \
    return st_;                               \
  }
  EXX_ALLOC(p->Gs, gbuf.size());
  EXX_ALLOC(p->tw, twbuf.size());
  if (!twzbuf.empty()) {
    EXX_ALLOC(p->twz, twzbuf.size());
  }
  EXX_ALLOC(p->d_occ, norb * sizeof(double));
  EXX_ALLOC(p->d_pairs, pairs.size() * sizeof(int4));
  EXX_ALLOC(p->epart, (size_t)p->maxpairs * nper * sizeof(double));
  EXX_ALLOC(p->Epair, (size_t)p->P * sizeof(double));
  EXX_ALLOC(p->X2, (size_t)p->maxpairs * m * n * (2 * nh) * cs);
  EXX_ALLOC(p->V, (size_t)p->maxpairs * n3 * rs);
  if (precision == EXX_FP32 && !(flags & EXX_FLAG_VX_FP64)) {
    EXX_ALLOC(p->vacc, (size_t)norb * n3 * sizeof(double));
  }
  EXX_ALLOC(p->E_dev, sizeof(double));
  EXX_ALLOC(p->d_err, 2 * sizeof(int));
  // pipeline lanes: two by default, one where the slab kernels run as CTA
  // clusters (512 orbitals on 160^3: 16.53 s per step with one lane, 16.59 s
  // with two); EXX_LANES=1..3 at plan creation chooses; never more than the
  // plan has tiles
  {
    const char* env = std::getenv("EXX_LANES");
    int nl = ops->clustered ? 1 : kDefaultLanes;
    if (env && env[0] >= '1' && env[0] <= '0' + kMaxLanes && env[1] == '\0') nl = env[0] - '0';
    p->max_lanes = p->lanes = (int)std::min<size_t>((size_t)nl, p->tiles.size());
  }
  for (int l = 1; l < p->max_lanes; ++l) {
    EXX_ALLOC(p->epx[l], (size_t)p->maxpairs * nper * sizeof(double));
    EXX_ALLOC(p->X2x[l], (size_t)p->maxpairs * m * n * (2 * nh) * cs);
    EXX_ALLOC(p->Vx[l], (size_t)p->maxpairs * n3 * rs);
  }
#undef EXX_ALLOC

  cudaError_t e = cudaMemcpyAsync(p->Gs, gbuf.data(), gbuf.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(p->tw, twbuf.data(), twbuf.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && p->twz)
    e = cudaMemcpyAsync(p->twz, twzbuf.data(), twzbuf.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(p->d_occ, p->occ.data(), norb * sizeof(double), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(p->d_pairs, pairs.data(), pairs.size() * sizeof(int4), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(p->Epair, 0, (size_t)p->P * sizeof(double), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(p->d_err, 0, 2 * sizeof(int), st);
  // test hook (EXX_TEST_STALL_TABLE_COPY=1): the staged kernel-table copy is
  // never issued, so its bounded wait runs out and exx_energy returns
  // EXX_ERR_TIMEOUT; the context stays usable
  if (e == cudaSuccess && ops->stage_table) {
    const char* hook = std::getenv("EXX_TEST_STALL_TABLE_COPY");
    if (hook != nullptr && hook[0] == '1') {
      static const int one = 1;
      e = cudaMemcpyAsync(p->d_err + 1, &one, sizeof(int), cudaMemcpyHostToDevice, st);
    }
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess && ops->stage_table && !exx::make_ktab_map(&p->gmap, p->Gs, nh, nz))
    e = cudaErrorInvalidValue;
  if (e == cudaSuccess) e = ops->setup();
  if (e == cudaSuccess && p->max_lanes > 1) {
    for (int l = 0; l < p->max_lanes && e == cudaSuccess; ++l) {
      e = cudaStreamCreateWithFlags(&p->ls[l], cudaStreamNonBlocking);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev_done[l], cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev_free[l], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    free_plan(p);
    delete p;
    return e == cudaErrorMemoryAllocation ? EXX_ERR_OOM : EXX_ERR_CUDA;
  }
  *out = p;
  return EXX_OK;
}

exx_status_t exx_plan_destroy(exx_plan_t p) {
  if (p == nullptr) return EXX_OK;
  free_plan(p);
  delete p;
  return EXX_OK;
}

exx_status_t exx_plan_info(exx_plan_t p, int* tile, int* ntiles, size_t* workspace_bytes,
                           int* launches_apply, int* launches_energy) {
  if (p == nullptr) return EXX_ERR_INVALID_ARG;
  int nt = 0;
  for (char m : p->mine) nt += m ? 1 : 0;
  if (tile) *tile = p->T;
  if (ntiles) *ntiles = nt;
  if (workspace_bytes) *workspace_bytes = p->ws;
  const bool conv = p->vacc != nullptr;
  if (launches_apply) *launches_apply = 5 * nt + 1 + (conv ? 1 : 0);
  if (launches_energy) *launches_energy = 3 * nt + 1;
  return EXX_OK;
}


// Host-buffer overlap (exx_apply_host): tiles wait for the input events of
// their two orbital blocks (recorded by the copy stream after each block's
// host-to-device copy), and when a tile row ends, the vx of its block is
// complete (row-major tiles bi <= bj: block b appears only in rows <= b), so
// it is converted and handed to the copy stream through ev_out[b].
struct HostOverlap {
  const std::vector<cudaEvent_t>* in;
  const std::vector<cudaEvent_t>* out;
};

// apply: also the inverse transforms and the accumulation into vxpsi, which
// receives (Vx psi)_k (grad = false) or dE_x/dpsi_k = 2 f_k h^3 (Vx psi)_k
// (grad = true).
static exx_status_t run(exx_plan_t p, const void* psi, void* vxpsi, double* E_dev, bool apply,
                        cudaStream_t st, const HostOverlap* ov = nullptr, bool grad = false) {
  const int n = p->n, N = p->N;
  const long long n3 = (long long)n * n * n;
  const double h3 = p->h * p->h * p->h;
  const int nper = (p->ops->n + 1) * p->ops->nyb;
  double* acc = nullptr;
  if (apply) {
    acc = p->vacc ? p->vacc : static_cast<double*>(vxpsi);
    EXX_CUDA(p, cudaMemsetAsync(acc, 0, (size_t)N * n3 * sizeof(double), st));
  }
  const double c = -p->alpha;
  const double gs = grad ? 2.0 * h3 : 0.0;
  if (p->sharded)  // pair energies of other ranks' tiles must read as zero
    EXX_CUDA(p, cudaMemsetAsync(p->Epair, 0, (size_t)p->P * sizeof(double), st));
  // Lanes: consecutive tiles go round-robin over the lanes' streams, each with
  // its own spectrum, potential and partial-energy buffers, so that the
  // transforms of one tile run beside those of the next; the accumulation
  // stays on the caller's stream in tile order (identical sums, no two updates
  // of one accumulator at a time), and a lane overwrites its V only after the
  // accumulation of its previous tile has read it.
  const int nl = p->lanes;
  if (nl > 1) {
    EXX_CUDA(p, cudaEventRecord(p->ev_fork, st));
    for (int l = 0; l < nl; ++l) EXX_CUDA(p, cudaStreamWaitEvent(p->ls[l], p->ev_fork, 0));
  }
  void* X2l[kMaxLanes];
  void* Vl[kMaxLanes];
  double* epl[kMaxLanes];
  bool used[kMaxLanes];
  int waited[kMaxLanes];  // per lane: input blocks 0..waited are known to have arrived
  for (int l = 0; l < kMaxLanes; ++l) {
    X2l[l] = l ? p->X2x[l] : p->X2;
    Vl[l] = l ? p->Vx[l] : p->V;
    epl[l] = l ? p->epx[l] : p->epart;
    used[l] = false;
    waited[l] = -1;
  }
  int k = 0;
  for (size_t ti = 0; ti < p->tiles.size(); ++ti) {
    if (!p->mine[ti]) continue;
    const Tile& t = p->tiles[ti];
    const int4* pr = p->d_pairs + t.off;
    const int l = nl > 1 ? (k++ % nl) : 0;
    cudaStream_t sl = nl > 1 ? p->ls[l] : st;
    void* X2 = X2l[l];
    void* Vt = Vl[l];
    double* ep = epl[l];
    if (ov) {
      const int bj = t.j0 / p->T;
      while (waited[l] < bj) EXX_CUDA(p, cudaStreamWaitEvent(sl, (*ov->in)[++waited[l]], 0));
    }
    {
      ProfScope ps(p, K_FWD, sl);
      p->ops->fwd_xy(psi, nullptr, pr, t.count, X2, p->tw, n3, sl);
    }
    {
      ProfScope ps(p, K_ZCONV, sl);
      p->ops->zconv(X2, p->Gs, p->twz ? p->twz : p->tw, &p->gmap, ep, p->d_err, t.count, !apply,
                    sl);
    }
    {
      ProfScope ps(p, K_PAIRE, sl);
      k_pair_energy<<<(t.count * 32 + 255) / 256, 256, 0, sl>>>(ep, nper, pr, t.count, h3,
                                                                  p->Epair);
    }
    if (apply) {
      if (nl > 1 && used[l]) EXX_CUDA(p, cudaStreamWaitEvent(sl, p->ev_free[l], 0));
      {
        ProfScope ps(p, K_INV, sl);
        p->ops->inv_yx(X2, Vt, p->tw, t.count, sl);
      }
      if (nl > 1) {
        EXX_CUDA(p, cudaEventRecord(p->ev_done[l], sl));
        EXX_CUDA(p, cudaStreamWaitEvent(st, p->ev_done[l], 0));
      }
      used[l] = true;
      ProfScope ps(p, K_ACCUM, st);
      // vector width: 4 (FP32) or 2 values per thread when n^3 and the
      // caller's pointers allow aligned vector accesses
      const bool al = ((uintptr_t)psi % 16 == 0) && ((uintptr_t)acc % 16 == 0);
      const bool v2 = al && (n3 % 2) == 0;
      const int mode = (t.ti == 8 && t.tj == 8) ? (t.diag ? 2 : 1) : 0;
      if (p->prec == EXX_FP64)
        launch_accum<double>(v2, mode, static_cast<const double*>(psi),
                             static_cast<const double*>(Vt), acc, p->d_occ, t, c, gs, n3, st);
      else
        launch_accum<float>(v2, mode, static_cast<const float*>(psi),
                            static_cast<const float*>(Vt), acc, p->d_occ, t, c, gs, n3, st);
      if (nl > 1) EXX_CUDA(p, cudaEventRecord(p->ev_free[l], st));
    }
    const bool row_end = ti + 1 == p->tiles.size() || p->tiles[ti + 1].i0 != t.i0;
    if (ov && apply && row_end) {
      const int b = t.i0 / p->T;
      if (p->vacc) {
        ProfScope ps(p, K_CONV, st);
        const long long cnt = (long long)t.ti * n3, off = (long long)t.i0 * n3;
        long long blocks = (cnt + 255) / 256;
        if (blocks > 152 * 32) blocks = 152 * 32;
        k_to_float<<<(int)blocks, 256, 0, st>>>(p->vacc + off, static_cast<float*>(vxpsi) + off, cnt);
      }
      EXX_CUDA(p, cudaEventRecord((*ov->out)[b], st));
    }
  }
  if (nl > 1)  // join: every lane's pair energies (and, for apply, V reads) are done
    for (int l = 0; l < nl; ++l) {
      EXX_CUDA(p, cudaEventRecord(p->ev_done[l], p->ls[l]));
      EXX_CUDA(p, cudaStreamWaitEvent(st, p->ev_done[l], 0));
    }
  {
    ProfScope ps(p, K_TOTAL, st);
    k_exx_total<<<1, 256, 0, st>>>(p->Epair, p->P, N, p->d_occ, p->alpha, E_dev ? E_dev : p->E_dev);
  }
  if (apply && p->vacc && !ov) {
    ProfScope ps(p, K_CONV, st);
    const long long tot = (long long)N * n3;
    long long blocks = (tot + 255) / 256;
    if (blocks > 152 * 32) blocks = 152 * 32;
    k_to_float<<<(int)blocks, 256, 0, st>>>(p->vacc, static_cast<float*>(vxpsi), tot);
  }
  EXX_CUDA(p, cudaGetLastError());
  return EXX_OK;
}

exx_status_t exx_apply_async(exx_plan_t p, const void* psi, void* vxpsi, double* E_dev,
                             void* cuda_stream) {
  if (p == nullptr || psi == nullptr || vxpsi == nullptr) return EXX_ERR_INVALID_ARG;
  return run(p, psi, vxpsi, E_dev, true, static_cast<cudaStream_t>(cuda_stream));
}

exx_status_t exx_gradient_async(exx_plan_t p, const void* psi, void* grad, double* E_dev,
                                void* cuda_stream) {
  if (p == nullptr || psi == nullptr || grad == nullptr) return EXX_ERR_INVALID_ARG;
  return run(p, psi, grad, E_dev, true, static_cast<cudaStream_t>(cuda_stream), nullptr, true);
}

exx_status_t exx_energy_async(exx_plan_t p, const void* psi, double* E_dev, void* cuda_stream) {
  if (p == nullptr || psi == nullptr) return EXX_ERR_INVALID_ARG;
  return run(p, psi, nullptr, E_dev, false, static_cast<cudaStream_t>(cuda_stream));
}

// A bounded device-side wait that ran out leaves a flag; the synchronising
// calls report it as EXX_ERR_TIMEOUT (and clear it).
static exx_status_t check_wait_flag(exx_plan_t p, cudaStream_t st) {
  int f = 0;
  EXX_CUDA(p, cudaMemcpyAsync(&f, p->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
  EXX_CUDA(p, cudaStreamSynchronize(st));
  if (f == 0) return EXX_OK;
  EXX_CUDA(p, cudaMemsetAsync(p->d_err, 0, sizeof(int), st));
  p->err = "a device-side wait ran out (kernel-table copy)";
  return EXX_ERR_TIMEOUT;
}

exx_status_t exx_apply(exx_plan_t p, const void* psi, void* vxpsi, double* E_out, void* cuda_stream) {
  if (p == nullptr || psi == nullptr || vxpsi == nullptr) return EXX_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  exx_status_t s = run(p, psi, vxpsi, nullptr, true, st);
  if (s != EXX_OK || E_out == nullptr) return s;
  EXX_CUDA(p, cudaMemcpyAsync(E_out, p->E_dev, sizeof(double), cudaMemcpyDeviceToHost, st));
  return check_wait_flag(p, st);
}

exx_status_t exx_gradient(exx_plan_t p, const void* psi, void* grad, double* E_out,
                          void* cuda_stream) {
  if (p == nullptr || psi == nullptr || grad == nullptr) return EXX_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  exx_status_t s = run(p, psi, grad, nullptr, true, st, nullptr, true);
  if (s != EXX_OK || E_out == nullptr) return s;
  EXX_CUDA(p, cudaMemcpyAsync(E_out, p->E_dev, sizeof(double), cudaMemcpyDeviceToHost, st));
  return check_wait_flag(p, st);
}

exx_status_t exx_energy(exx_plan_t p, const void* psi, double* E_out, void* cuda_stream) {
  if (p == nullptr || psi == nullptr || E_out == nullptr) return EXX_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  exx_status_t s = run(p, psi, nullptr, nullptr, false, st);
  if (s != EXX_OK) return s;
  EXX_CUDA(p, cudaMemcpyAsync(E_out, p->E_dev, sizeof(double), cudaMemcpyDeviceToHost, st));
  return check_wait_flag(p, st);
}

// exx_apply_host / exx_gradient_host: orbitals and results in host memory
static exx_status_t run_host(exx_plan_t p, const void* psi_host, void* vxpsi_host, double* E_out,
                             void* cuda_stream, bool grad) {
  if (p == nullptr || psi_host == nullptr || vxpsi_host == nullptr) return EXX_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const size_t cnt = (size_t)p->N * p->n * p->n * p->n;
  const size_t ps = p->prec == EXX_FP64 ? sizeof(double) : sizeof(float);
  const size_t vs = (p->prec == EXX_FP64 || (p->flags & EXX_FLAG_VX_FP64)) ? sizeof(double) : sizeof(float);
  if (p->h_psi == nullptr) {
    exx_status_t s = dalloc(p, &p->h_psi, cnt * ps);
    if (s != EXX_OK) return s;
  }
  if (p->h_vx == nullptr) {
    exx_status_t s = dalloc(p, &p->h_vx, cnt * vs);
    if (s != EXX_OK) return s;
  }
  if (p->sharded) {  // partial results: one copy each way around the pipeline
    EXX_CUDA(p, cudaMemcpyAsync(p->h_psi, psi_host, cnt * ps, cudaMemcpyHostToDevice, st));
    exx_status_t s = run(p, p->h_psi, p->h_vx, nullptr, true, st, nullptr, grad);
    if (s != EXX_OK) return s;
    EXX_CUDA(p, cudaMemcpyAsync(vxpsi_host, p->h_vx, cnt * vs, cudaMemcpyDeviceToHost, st));
    if (E_out) EXX_CUDA(p, cudaMemcpyAsync(E_out, p->E_dev, sizeof(double), cudaMemcpyDeviceToHost, st));
    return check_wait_flag(p, st);
  }
  // copies per orbital block on a second stream, overlapped with the tiles:
  // block b goes in ahead of the first tile that reads it, and its vx goes
  // out as soon as the last tile row that touches it has finished
  const int nb = (p->N + p->T - 1) / p->T;
  if (p->cst == nullptr)
    EXX_CUDA(p, cudaStreamCreateWithFlags(&p->cst, cudaStreamNonBlocking));
  auto mk = [&](cudaEvent_t* e) { return cudaEventCreateWithFlags(e, cudaEventDisableTiming); };
  if (p->ev_start == nullptr) EXX_CUDA(p, mk(&p->ev_start));
  if (p->ev_join == nullptr) EXX_CUDA(p, mk(&p->ev_join));
  while ((int)p->ev_in.size() < nb) {
    cudaEvent_t a, b;
    EXX_CUDA(p, mk(&a));
    p->ev_in.push_back(a);
    EXX_CUDA(p, mk(&b));
    p->ev_out.push_back(b);
  }
  const size_t blk = (size_t)p->T * p->n * p->n * p->n;  // elements per orbital block
  EXX_CUDA(p, cudaEventRecord(p->ev_start, st));  // earlier work on st is done first
  EXX_CUDA(p, cudaStreamWaitEvent(p->cst, p->ev_start, 0));
  for (int b = 0; b < nb; ++b) {
    const size_t off = (size_t)b * blk, len = std::min(blk, cnt - off);
    EXX_CUDA(p, cudaMemcpyAsync(static_cast<char*>(p->h_psi) + off * ps,
                                static_cast<const char*>(psi_host) + off * ps, len * ps,
                                cudaMemcpyHostToDevice, p->cst));
    EXX_CUDA(p, cudaEventRecord(p->ev_in[b], p->cst));
  }
  HostOverlap ov{&p->ev_in, &p->ev_out};
  exx_status_t s = run(p, p->h_psi, p->h_vx, nullptr, true, st, &ov, grad);
  if (s != EXX_OK) {
    cudaStreamSynchronize(p->cst);
    return s;
  }
  for (int b = 0; b < nb; ++b) {
    const size_t off = (size_t)b * blk, len = std::min(blk, cnt - off);
    EXX_CUDA(p, cudaStreamWaitEvent(p->cst, p->ev_out[b], 0));
    EXX_CUDA(p, cudaMemcpyAsync(static_cast<char*>(vxpsi_host) + off * vs,
                                static_cast<const char*>(p->h_vx) + off * vs, len * vs,
                                cudaMemcpyDeviceToHost, p->cst));
  }
  if (E_out) EXX_CUDA(p, cudaMemcpyAsync(E_out, p->E_dev, sizeof(double), cudaMemcpyDeviceToHost, st));
  EXX_CUDA(p, cudaEventRecord(p->ev_join, p->cst));
  EXX_CUDA(p, cudaStreamWaitEvent(st, p->ev_join, 0));
  return check_wait_flag(p, st);
}

exx_status_t exx_apply_host(exx_plan_t p, const void* psi_host, void* vxpsi_host, double* E_out,
                            void* cuda_stream) {
  return run_host(p, psi_host, vxpsi_host, E_out, cuda_stream, false);
}

exx_status_t exx_gradient_host(exx_plan_t p, const void* psi_host, void* grad_host, double* E_out,
                               void* cuda_stream) {
  return run_host(p, psi_host, grad_host, E_out, cuda_stream, true);
}

exx_status_t exx_plan_set_lanes(exx_plan_t p, int lanes) {
  if (p == nullptr || lanes < 1 || lanes > kMaxLanes) return EXX_ERR_INVALID_ARG;
  if (lanes > p->max_lanes) return EXX_ERR_NOT_SUPPORTED;
  p->lanes = lanes;
  return EXX_OK;
}

exx_status_t exx_plan_get_lanes(exx_plan_t p, int* lanes) {
  if (p == nullptr || lanes == nullptr) return EXX_ERR_INVALID_ARG;
  *lanes = p->lanes;
  return EXX_OK;
}

exx_status_t exx_profile_enable(exx_plan_t p, int enable) {
  if (p == nullptr) return EXX_ERR_INVALID_ARG;
  p->prof = enable != 0;
  return EXX_OK;
}

exx_status_t exx_profile_read(exx_plan_t p, double* ms, long long* launches, int reset) {
  if (p == nullptr) return EXX_ERR_INVALID_ARG;
  for (int k = 0; k < EXX_NKINDS; ++k) {
    for (size_t u = 0; u < p->used[k]; ++u) {
      float t = 0.0f;
      EXX_CUDA(p, cudaEventSynchronize(p->ev[k][2 * u + 1]));
      EXX_CUDA(p, cudaEventElapsedTime(&t, p->ev[k][2 * u], p->ev[k][2 * u + 1]));
      p->ms[k] += t;
      p->cnt[k] += 1;
    }
    p->used[k] = 0;
    if (ms) ms[k] = p->ms[k];
    if (launches) launches[k] = p->cnt[k];
    if (reset) {
      p->ms[k] = 0.0;
      p->cnt[k] = 0;
    }
  }
  return EXX_OK;
}

exx_status_t exx_shard_tiles(int norb, int tile, int nranks, int* desc_out, int* owner_out,
                             int* ntiles) {
  if (norb < 1 || nranks < 1 || tile < 0 || tile > 8 || ntiles == nullptr) return EXX_ERR_INVALID_ARG;
  const std::vector<Tile> tiles = make_tiles(norb, default_tile(norb, tile));
  *ntiles = (int)tiles.size();
  if (desc_out)
    for (size_t k = 0; k < tiles.size(); ++k) {
      desc_out[5 * k + 0] = tiles[k].i0;
      desc_out[5 * k + 1] = tiles[k].ti;
      desc_out[5 * k + 2] = tiles[k].j0;
      desc_out[5 * k + 3] = tiles[k].tj;
      desc_out[5 * k + 4] = tiles[k].diag;
    }
  if (owner_out) {
    const std::vector<int> own = shard_owners(tiles, nranks);
    for (size_t k = 0; k < own.size(); ++k) owner_out[k] = own[k];
  }
  return EXX_OK;
}

exx_status_t exx_plan_set_shard(exx_plan_t p, int rank, int nranks) {
  if (p == nullptr || nranks < 1 || rank < 0 || rank >= nranks) return EXX_ERR_INVALID_ARG;
  const std::vector<int> own = shard_owners(p->tiles, nranks);
  for (size_t k = 0; k < own.size(); ++k) p->mine[k] = (own[k] == rank);
  p->sharded = nranks > 1;
  return EXX_OK;
}

exx_status_t exx_pair_energies(exx_plan_t p, double* out_host, void* cuda_stream) {
  if (p == nullptr || out_host == nullptr) return EXX_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  EXX_CUDA(p, cudaMemcpyAsync(out_host, p->Epair, (size_t)p->P * sizeof(double),
                              cudaMemcpyDeviceToHost, st));
  EXX_CUDA(p, cudaStreamSynchronize(st));
  return EXX_OK;
}

}  // extern "C"
