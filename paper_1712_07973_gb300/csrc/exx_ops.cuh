// Per-grid-size launch table of the pair pipeline.  One OpsImpl<R, N, ...> is
// instantiated per supported (precision, n, boundary conditions) in the
// exx_inst_*.cu files; the C-ABI layer picks the table at plan creation.
#pragma once

#include <cmath>
#include <cstddef>

#include <cuda.h>
#include <cudaTypedefs.h>

#include "exx_gain.cuh"
#include "exx_kernels.cuh"
#include "exx_persist.cuh"

namespace exx {

struct Ops {
  int n = 0;         // half the line length of the x and y transforms (line 2n)
  int nz = 0;        // half the line length of the z transform (= n unless mixed)
  int grid = 0;      // grid points per axis: n (free BC) or 2n (periodic)
  bool periodic = false;    // x and y periodic
  bool periodic_z = false;  // z periodic
  bool supported = false;
  int nyb = 0;             // zconv column blocks per kx plane
  int nt_a = 0, nt_c = 0;  // threads per CTA of fwd_xy / inv_yx
  int nw_b = 0;            // warps per CTA of zconv
  size_t smem_a = 0, smem_b = 0, smem_c = 0;
  cudaError_t (*setup)() = nullptr;
  // energy gains of the FP32 forward transforms (null for FP64): gx[n+1],
  // gy[2n], gz[2nz]
  void (*gains)(double* gx, double* gy, double* gz) = nullptr;
  bool table_fold_y = false;  // kernel-table layout (build_kernel_table)
  bool clustered = false;     // slab kernels launched as CTA clusters
  // psi_tab (device array of orbital-array pointers, indexed by the pair's
  // molecule slot) may be null, in which case every pair reads psi
  void (*fwd_xy)(const void* psi, const void* const* psi_tab, const int4* pairs, int npair,
                 void* X, const void* tw, long long n3, cudaStream_t st) = nullptr;
  // gmap: TMA descriptor of the kernel table (make_ktab_map; read only when
  // stage_table); err: two device ints, [0] set by a wait that ran out, [1] a
  // test hook that makes the staged copy's wait run out
  void (*zconv)(void* X, const void* Gs, const void* tw, const CUtensorMap* gmap, double* epart,
                int* err, int npair, bool energy_only, cudaStream_t st) = nullptr;
  bool stage_table = false;
  void (*inv_yx)(const void* X3, void* V, const void* tw, int npair, cudaStream_t st) = nullptr;
  // persistent batched kernel (FP32, free boundary conditions, slab kernels
  // without clusters): threads per CTA, and the launch of a queue
  bool persist_ok = false;
  int persist_nt = 0;
  cudaError_t (*persist)(const PersistArgs& a, cudaStream_t st) = nullptr;
};

constexpr size_t kSmemPerCTA = 227 * 1024 - 256;  // largest dynamic allocation of one CTA

// Launch shape of the slab kernels (fwd_xy, inv_yx): shared memory = fixed
// part (slab + twiddles) + y-pass scratch.  In order of preference:
//   warp-owned y passes (q = 0, two scratch rows per warp) as four CTAs of
//   192 threads per SM when asked for and they fit in a quarter of an SM
//   (small slabs: periodic 96^3 -6.6% per exx_apply against two CTAs of 320
//   with 160 threads per CTA, a further -1.8% with 192),
//   two CTAs of 320 when they fit in half an SM, else one CTA of 640;
//   FP32: the slab split over a four-CTA cluster (cl = 4, a quarter of the
//   columns per CTA; fixed4 is its fixed part) as two CTAs of 320 per SM;
//   the slab split over a two-CTA cluster (cl = 2, half the columns per CTA;
//   fixed2 is its fixed part), when allowed, with 640 or else 320 threads per
//   CTA; over a four-CTA cluster with 320 threads (FP64 n = 160);
//   CTA-wide batches of q rows.
// Measured at n = 96 (64 orbitals): warp-owned y passes with two CTAs per SM
// take fwd_xy from 13.3 to 13.0 ms and inv_yx from 13.5 to 11.1 ms per
// exx_apply.
struct SlabShape {
  int q, nt, minb, cl;
  size_t smem;
  bool fits;
};
constexpr SlabShape slab_shape(size_t fixed, size_t fixed2, bool split_ok, size_t line,
                               bool prefer_two, bool fp32, size_t fixed4 = 0,
                               bool split4_ok = false) {
  const size_t half = 113 * 1024;
  if (prefer_two && fp32 && fixed + 12 * line <= 56 * 1024)  // small slabs: four CTAs of 192
    return SlabShape{0, 192, 4, 1, fixed + 12 * line, true};
  if (prefer_two && fixed + 10 * line <= 56 * 1024)  // (FP64: 160, within the registers)
    return SlabShape{0, 160, 4, 1, fixed + 10 * line, true};
  if (prefer_two && fixed + 20 * line <= half) return SlabShape{0, 320, 2, 1, fixed + 20 * line, true};
  if (fixed + 40 * line <= kSmemPerCTA) return SlabShape{0, 640, 1, 1, fixed + 40 * line, true};
  // FP32 slabs beyond one SM (n = 160): four-CTA clusters of 320 threads, two
  // CTAs per SM, so that one CTA's transform phases overlap the other's memory
  // phases (a two-CTA cluster of 640 threads holds a whole SM)
  if (fp32 && split4_ok && fixed4 + 20 * line <= half)
    return SlabShape{0, 320, 2, 4, fixed4 + 20 * line, true};
  if (split_ok && fixed2 + 40 * line <= kSmemPerCTA)
    return SlabShape{0, 640, 1, 2, fixed2 + 40 * line, true};
  if (split_ok && fixed2 + 20 * line <= kSmemPerCTA)  // e.g. FP64 n = 128
    return SlabShape{0, 320, 1, 2, fixed2 + 20 * line, true};
  if (split4_ok && fixed4 + 20 * line <= kSmemPerCTA)  // FP64 n = 160
    return SlabShape{0, 320, 1, 4, fixed4 + 20 * line, true};
  if (prefer_two && fixed + 8 * line <= half) {
    size_t q = (half - fixed) / line;
    q = q > 32 ? 32 : q;
    return SlabShape{(int)q, 320, 2, 1, fixed + q * line, true};
  }
  if (fixed + line > kSmemPerCTA) return SlabShape{1, 640, 1, 1, fixed + line, false};
  size_t q = (kSmemPerCTA - fixed) / line;
  q = q > 64 ? 64 : q;
  return SlabShape{(int)q, 640, 1, 1, fixed + q * line, true};
}

// TMA descriptor of an FP32 zconv kernel table Gt[kx][kz][ky] (unfolded layout,
// kx <= n, kz < 2nz, ky < 2n): 3-D, box of min(2n, 32) ky by 2nz kz by one kx,
// no swizzle, out-of-range elements read as zero.  The driver's encoder is
// reached through the runtime (no link against the driver library).
inline bool make_ktab_map(CUtensorMap* map, const void* table, int n, int nz) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (encode == nullptr) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || fn == nullptr)
      return false;
    encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  const cuuint64_t L = 2 * (cuuint64_t)n, LZ = 2 * (cuuint64_t)nz;
  const cuuint64_t dims[3] = {L, LZ, (cuuint64_t)n + 1};
  const cuuint64_t strides[2] = {L * sizeof(float), L * LZ * sizeof(float)};
  const cuuint32_t box[3] = {(cuuint32_t)(L < 32 ? L : 32), (cuuint32_t)LZ, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  return encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void*>(table), dims, strides,
                box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Launch of a slab kernel; CL > 1 launches (CL, 1, 1) thread-block clusters.
template <int CL, typename... KArgs, typename... Args>
inline void launch_slab(void (*kern)(KArgs...), dim3 grid, int nt, size_t smem, cudaStream_t st,
                        Args... args) {
  if constexpr (CL == 1) {
    kern<<<grid, nt, smem, st>>>(args...);
  } else {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(nt);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = CL;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kern, args...);
  }
}

// zconv warps: a count that divides the L2-long passes when possible (12 for
// L2 = 12 measured 4% faster than 6 at n = 96)
constexpr int zconv_warps(int l2) {
  return (l2 % 8 == 0) ? 8 : (l2 % 6 == 0) ? 12 : (l2 % 10 == 0) ? 10 : (l2 % 7 == 0) ? 7
       : (l2 % 5 == 0) ? 5 : 4;
}

// Twiddle tables of one grid size, packed in one array of complex values
// rounded to nearest in the plan's precision; exponent e stands for
// w^e = exp(-2 pi i e / L), L = 2n:
//   [0, L)          w^k
//   [L, 2L)         TY[k1][n2] = w^(n2 k1), k1 < L1, n2 < L2
//   [2L, 2L+n)      TX[k1][n2] = w^(2 n2 k1), k1 < X1, n2 < X2
//   [2L+n, 3L+n)    TI[m2][k1] = w^(m2 k1), m2 < L2, k1 < L1
// The two-dimensional tables put the index that varies across the lanes of
// the slab kernels' passes fastest, so that their reads are conflict free.
inline size_t twiddle_count(int n) { return (size_t)7 * n; }
template <typename R> void build_twiddles(int n, R* out) {
  const int L = 2 * n, L1 = split_l1(L), L2 = L1 ? L / L1 : 1;
  const int X1 = split_x(n), X2 = X1 ? n / X1 : 1;
  auto put = [&](size_t idx, long e) {
    const double a = -M_PI * (double)(e % L) / (double)n;
    out[2 * idx] = (R)std::cos(a);
    out[2 * idx + 1] = (R)std::sin(a);
  };
  for (int k = 0; k < L; ++k) put(k, k);
  for (int k1 = 0; k1 < L1; ++k1)
    for (int n2 = 0; n2 < L2; ++n2) put(L + k1 * L2 + n2, (long)n2 * k1);
  for (int k1 = 0; k1 < X1; ++k1)
    for (int n2 = 0; n2 < X2; ++n2) put(2 * L + k1 * X2 + n2, (long)2 * n2 * k1);
  for (int m2 = 0; m2 < L2; ++m2)
    for (int k1 = 0; k1 < L1; ++k1) put(2 * L + n + m2 * L1 + k1, (long)m2 * k1);
}

// Kernel table of zconv (layout in exx_kernels.cuh) from the octant
// Ghat[kz][ky][kx], kz <= nz, kx, ky <= n: scale * Ghat / (gx[kx] gy[ky] gz[kz]),
// or with fold_y (nz = n only) the ky-folded rows without gy[ky] followed by
// 1 / gy[ky].  gx, gy, gz are the energy gains |d|^2 of the FP32 forward
// transforms (exx_gain.cuh), null for FP64.
inline size_t kernel_table_bytes(int n, int nz, size_t real_size, bool fold_y) {
  if (fold_y) return ktab_cy_offset(n, real_size) + 2 * (size_t)n * sizeof(double);
  return (size_t)(n + 1) * (2 * (size_t)nz) * (2 * (size_t)n) * real_size;
}
template <typename R>
void build_kernel_table(int n, int nz, bool fold_y, const double* octant, double scale,
                        const double* gx, const double* gy, const double* gz, unsigned char* out) {
  const size_t m = (size_t)n + 1, L = 2 * (size_t)n, LZ = 2 * (size_t)nz, row = fold_y ? m : L;
  R* G = reinterpret_cast<R*>(out);
  for (size_t kx = 0; kx < m; ++kx)
    for (size_t kz = 0; kz < LZ; ++kz) {
      const size_t kzf = kz <= (size_t)nz ? kz : LZ - kz;
      const double c = scale / ((gx ? gx[kx] : 1.0) * (gz ? gz[kz] : 1.0));
      for (size_t ky = 0; ky < row; ++ky) {
        const size_t kyf = ky <= (size_t)n ? ky : L - ky;
        const double cy = (fold_y || !gy) ? 1.0 : 1.0 / gy[ky];
        G[(kx * LZ + kz) * row + ky] = (R)(c * cy * octant[(kzf * m + kyf) * m + kx]);
      }
    }
  if (fold_y) {
    double* cy = reinterpret_cast<double*>(out + ktab_cy_offset(n, sizeof(R)));
    for (size_t k = 0; k < L; ++k) cy[k] = gy ? 1.0 / gy[k] : 1.0;
  }
}

// (N, PER): the x and y transforms; (NZ, PERZ): the z transform (mixed
// boundary conditions: slab = periodic x, y with free z; wire = the reverse).
template <typename R, int N, bool PER = false, int NZ = N, bool PERZ = PER> struct OpsImpl {
  using C = cplx<R>;
  static constexpr int G = PER ? 2 * N : N;  // grid points per axis
  static constexpr bool mixed = NZ != N || PERZ != PER;
  static_assert(G == (PERZ ? 2 * NZ : NZ), "one grid size on all axes");
  static constexpr int L = 2 * N;
  static constexpr int L1 = split_l1(L);
  static constexpr int L2 = L1 ? L / L1 : 1;
  static constexpr int LZ = 2 * NZ;
  static constexpr int LZ1 = split_z(LZ);
  static constexpr int LZ2 = LZ1 ? LZ / LZ1 : 1;
  static constexpr int X1 = split_x(N);
  static constexpr size_t slab = X1 ? (size_t)slab_elems(N, G) * sizeof(C) : 0;
  // two-CTA split: half the columns per CTA (the y-pass index split must fall
  // on a whole number of length-L2 groups)
  static constexpr bool split_ok = X1 && L1 && G % 2 == 0 && (G / 2) % L2 == 0;
  static constexpr size_t slab2 = split_ok ? (size_t)slab_elems(N, G / 2) * sizeof(C) : 0;
  // four-CTA split: a quarter of the columns per CTA
  static constexpr bool split4_ok = X1 && L1 && G % 4 == 0 && (G / 4) % L2 == 0;
  static constexpr size_t slab4 = split4_ok ? (size_t)slab_elems(N, G / 4) * sizeof(C) : 0;
  static constexpr size_t line = (size_t)((L2 * (L1 + 1)) | 1) * sizeof(C);
  static constexpr SlabShape SA = slab_shape(slab + (size_t)(L + N) * sizeof(C),
                                             slab2 + (size_t)(L + N) * sizeof(C), split_ok, line,
                                             true, sizeof(R) == 4,
                                             slab4 + (size_t)(L + N) * sizeof(C), split4_ok);
  static constexpr SlabShape SC = slab_shape(slab + (size_t)2 * L * sizeof(C),
                                             slab2 + (size_t)2 * L * sizeof(C), split_ok, line,
                                             true, sizeof(R) == 4,
                                             slab4 + (size_t)2 * L * sizeof(C), split4_ok);
  static constexpr int QA = SA.q, NT_A = SA.nt, MINB_A = SA.minb, CL_A = SA.cl;
  static constexpr int QC = SC.q, NT_C = SC.nt, MINB_C = SC.minb, CL_C = SC.cl;
  static constexpr size_t smem_a = SA.smem, smem_c = SC.smem;
  // FP32 z lines of L2 = 6 (96 points: periodic and wire 96^3, free 48^3): six
  // warps, so that each pass-1 and pass-3 unit has its own warp, and six CTAs
  // per SM (periodic 96^3 -3.3%, wire -9% per exx_apply against 12 warps)
  // (FP32 L2 = 14, 224-point lines: eight warps, two rounds in every pass,
  // rather than seven with three rounds in the second; FP32 L2 = 12,
  // 192-point lines: eight warps with the kernel table read from L2, four
  // CTAs per SM, -2.3% zconv at 96^3 against twelve warps with the staged
  // table at three CTAs)
  // (FP32 320-point lines of free 160^3, split 20 x 16 (split_z): ten warps, two
  // CTAs per SM; 16 columns per CTA with two units per warp, five warps and
  // four CTAs per SM, measured 7% slower)
  static constexpr int NW = (sizeof(R) == 4 && LZ1 == 20)   ? 10  // 320-point lines (split_z)
                            : (sizeof(R) == 4 && LZ2 == 6)  ? 6
                            : (sizeof(R) == 4 && LZ2 == 14) ? 8
                            : (sizeof(R) == 4 && LZ2 == 12) ? 8
                                                            : zconv_warps(LZ2);
  static constexpr int W = L < 32 ? L : 32;
  static constexpr int NYB = (L + W - 1) / W;
  // zconv: twiddles + column buffer, plus the staged kernel-table slice when
  // its rows are 16-byte aligned and three CTAs (the FP32 launch bound) still
  // fit in an SM's 228 KB of shared memory
  static constexpr size_t smem_b0 = ((size_t)LZ + (size_t)LZ * W) * sizeof(C);
  static constexpr size_t smem_g = (size_t)LZ * W * sizeof(R);
  static constexpr size_t smem_bg = zconv_gsm_offset(LZ, W, sizeof(C)) + smem_g + 128;  // + alignment slack
  static constexpr bool stage_g = sizeof(R) == 4 && LZ2 != 12 && (W * sizeof(R)) % 16 == 0 &&
                                  (L * sizeof(R)) % 16 == 0 && LZ <= 256 &&
                                  3 * (smem_bg + 1024) <= 228 * 1024;
  static constexpr size_t smem_b = stage_g ? smem_bg : smem_b0;
  // CTAs per SM the zconv register budget is sized for (FP32): as many as
  // shared memory allows, at least three and at most eight; else two
  static constexpr int CTAS_B = (int)((228 * 1024) / (smem_b + 1024));
  static constexpr int MINB_B = (sizeof(R) == 4 && CTAS_B >= 3) ? (CTAS_B < 8 ? CTAS_B : 8)
                                : CTAS_B >= 2 ? 2 : 1;
  // ky-folded kernel table where the unfolded one would exceed 24 MB
  static constexpr bool fold_y = !mixed && !stage_g && (size_t)(N + 1) * (2 * N) * (2 * N) * sizeof(R) > (24u << 20);
  static constexpr bool ok = L1 != 0 && LZ1 != 0 && X1 != 0 && SA.fits && SC.fits && smem_b <= kSmemPerCTA;
  template <bool EO> static constexpr auto zk() {
    return &k_zconv<R, N, NW, MINB_B, stage_g, fold_y, PER, EO, NZ, PERZ>;
  }
  // persistent batched kernel: the slab kernels' CTA shape (one per SM share),
  // shared memory for the largest pass
  static constexpr bool persist_ok = sizeof(R) == 4 && !PER && !mixed && ok && QA == 0 &&
                                     QC == 0 && CL_A == 1 && CL_C == 1 && NT_A == NT_C;
  static constexpr int NT_P = NT_A;
  static constexpr int MINB_P = MINB_A < MINB_C ? MINB_A : MINB_C;
  static constexpr size_t smem_p = smem_a > smem_c ? (smem_a > smem_b0 ? smem_a : smem_b0)
                                                   : (smem_c > smem_b0 ? smem_c : smem_b0);
  static constexpr auto pk() { return &k_persist<N, NT_P, MINB_P, fold_y>; }
  static cudaError_t persist(const PersistArgs& a, cudaStream_t st) {
    if constexpr (persist_ok) {
      static int grid = 0;  // resident CTAs on this device
      if (grid == 0) {
        int dev = 0, sms = 0, per = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(pk(), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_p);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, pk(), NT_P, smem_p);
        if (e != cudaSuccess) return e;
        grid = (per > 0 ? per : 1) * sms;
      }
      if (a.total <= 0) return cudaSuccess;  // set-up only (before any capture)
      const int g = a.total < grid ? a.total : grid;
      pk()<<<g > 0 ? g : 1, NT_P, smem_p, st>>>(a);
      return cudaGetLastError();
    }
    return cudaErrorNotSupported;
  }

  // gains of the x and y transforms, and of the z transform
  static void gains(double* gx, double* gy, double* gz) {
    GainModel<N, PER>::gains(gx, gy);
    if constexpr (!mixed && LZ1 == L1) {
      for (int k = 0; k < L; ++k) gz[k] = gy[k];
    } else {  // the z line differs from the y line in length, periodicity or split
      double tx[NZ + 1];
      GainModel<NZ, PERZ, F32c, LZ1>::gains(tx, gz);
    }
  }

  static cudaError_t setup() {
    if constexpr (ok) {
      cudaError_t e;
      e = cudaFuncSetAttribute(k_fwd_xy<R, N, NT_A, MINB_A, QA, CL_A, PER>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_a);
      if (e != cudaSuccess) return e;
      e = cudaFuncSetAttribute(zk<false>(), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_b);
      if (e != cudaSuccess) return e;
      e = cudaFuncSetAttribute(zk<true>(), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_b);
      if (e != cudaSuccess) return e;
      return cudaFuncSetAttribute(k_inv_yx<R, N, NT_C, MINB_C, QC, CL_C, PER>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_c);
    }
    return cudaErrorNotSupported;
  }
  static void fwd_xy(const void* psi, const void* const* psi_tab, const int4* pairs, int npair,
                     void* X, const void* tw, long long n3, cudaStream_t st) {
    if constexpr (ok)
      launch_slab<CL_A>(k_fwd_xy<R, N, NT_A, MINB_A, QA, CL_A, PER>, dim3(CL_A * npair, G), NT_A,
                        smem_a, st, static_cast<const R*>(psi),
                        reinterpret_cast<const R* const*>(psi_tab), pairs, static_cast<C*>(X),
                        static_cast<const C*>(tw), n3);
  }
  static void zconv(void* X, const void* Gs, const void* tw, const CUtensorMap* gmap,
                    double* epart, int* err, int npair, bool energy_only, cudaStream_t st) {
    if constexpr (ok) {
      const dim3 grid(NYB, npair, N + 1);
      CUtensorMap m{};
      if (stage_g && gmap) m = *gmap;
      if (energy_only)
        zk<true>()<<<grid, 32 * NW, smem_b, st>>>(static_cast<C*>(X), static_cast<const R*>(Gs),
                                                  static_cast<const C*>(tw), epart, m, err);
      else
        zk<false>()<<<grid, 32 * NW, smem_b, st>>>(static_cast<C*>(X), static_cast<const R*>(Gs),
                                                   static_cast<const C*>(tw), epart, m, err);
    }
  }
  static void inv_yx(const void* X, void* V, const void* tw, int npair, cudaStream_t st) {
    if constexpr (ok)
      launch_slab<CL_C>(k_inv_yx<R, N, NT_C, MINB_C, QC, CL_C, PER>, dim3(G * CL_C, npair), NT_C,
                        smem_c, st, static_cast<const C*>(X), static_cast<R*>(V),
                        static_cast<const C*>(tw));
  }
  static Ops make() {
    Ops o;
    o.n = N;
    o.nz = NZ;
    o.grid = G;
    o.periodic = PER;
    o.periodic_z = PERZ;
    o.supported = ok;
    o.nyb = NYB;
    o.nt_a = NT_A;
    o.nt_c = NT_C;
    o.nw_b = NW;
    o.smem_a = smem_a;
    o.smem_b = smem_b;
    o.smem_c = smem_c;
    o.setup = &setup;
    o.table_fold_y = fold_y;
    o.clustered = CL_A > 1 || CL_C > 1;
    o.stage_table = stage_g;
    if constexpr (ok && sizeof(R) == 4) o.gains = &gains;
    o.fwd_xy = &fwd_xy;
    o.zconv = &zconv;
    o.inv_yx = &inv_yx;
    o.persist_ok = persist_ok;
    o.persist_nt = NT_P;
    if constexpr (persist_ok) o.persist = &persist;
    return o;
  }
};

}  // namespace exx

// periodic boundary conditions on a grid of 2N points per axis
#define EXX_DEFINE_OPS_PER(N)                                       \
  namespace exx {                                                   \
  const Ops* ops_pf32_##N() {                                       \
    static const Ops o = OpsImpl<float, N, true>::make();           \
    return &o;                                                      \
  }                                                                 \
  const Ops* ops_pf64_##N() {                                       \
    static const Ops o = OpsImpl<double, N, true>::make();          \
    return &o;                                                      \
  }                                                                 \
  }

// slab (x, y periodic, z free) on a grid of 2N points per axis, and wire
// (x, y free, z periodic) on a grid of N points per axis (N even)
#define EXX_DEFINE_OPS_SLAB(N)                                      \
  namespace exx {                                                   \
  const Ops* ops_sf32_##N() {                                       \
    static const Ops o = OpsImpl<float, N, true, 2 * N, false>::make(); \
    return &o;                                                      \
  }                                                                 \
  const Ops* ops_sf64_##N() {                                       \
    static const Ops o = OpsImpl<double, N, true, 2 * N, false>::make(); \
    return &o;                                                      \
  }                                                                 \
  }
#define EXX_DEFINE_OPS_WIRE(N)                                      \
  namespace exx {                                                   \
  const Ops* ops_wf32_##N() {                                       \
    static const Ops o = OpsImpl<float, N, false, N / 2, true>::make(); \
    return &o;                                                      \
  }                                                                 \
  const Ops* ops_wf64_##N() {                                       \
    static const Ops o = OpsImpl<double, N, false, N / 2, true>::make(); \
    return &o;                                                      \
  }                                                                 \
  }

#define EXX_DEFINE_OPS(N)                                           \
  namespace exx {                                                   \
  const Ops* ops_f32_##N() {                                        \
    static const Ops o = OpsImpl<float, N>::make();                 \
    return &o;                                                      \
  }                                                                 \
  const Ops* ops_f64_##N() {                                        \
    static const Ops o = OpsImpl<double, N>::make();                \
    return &o;                                                      \
  }                                                                 \
  }
