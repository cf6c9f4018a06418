// Per-grid-size launch table of the pair pipeline.  One OpsImpl<R, N> is
// instantiated per supported (precision, n) in the exx_inst_*.cu files; the
// C-ABI layer picks the table at plan creation.
#pragma once

#include <cstddef>

#include "exx_kernels.cuh"

namespace exx {

struct Ops {
  int n = 0;
  bool supported = false;
  int nyb = 0;             // zconv column blocks per kx plane
  int nt_a = 0, nt_c = 0;  // threads per CTA of fwd_xy / inv_yx
  int nw_b = 0;            // warps per CTA of zconv
  size_t smem_a = 0, smem_b = 0, smem_c = 0;
  cudaError_t (*setup)() = nullptr;
  void (*fwd_xy)(const void* psi, const int4* pairs, int npair, void* X2, const void* tw,
                 long long n3, cudaStream_t st) = nullptr;
  void (*zconv)(void* X, const void* Gs, const void* tw, double* epart, int npair,
                bool energy_only, cudaStream_t st) = nullptr;
  void (*inv_yx)(const void* X3, void* V, const void* tw, int npair, cudaStream_t st) = nullptr;
};

constexpr size_t kSmemBudget = 227 * 1024 - 1024;  // per CTA, minus static shared

// largest batch (<= 16 lines) whose scratch fits next to the slab
constexpr int choose_q(size_t fixed, size_t per) {
  if (fixed >= kSmemBudget) return 0;
  size_t q = (kSmemBudget - fixed) / per;
  return q > 16 ? 16 : (int)q;
}

template <typename R, int N> struct OpsImpl {
  using C = cplx<R>;
  static constexpr int L = 2 * N;
  static constexpr int L1 = split_l1(L);
  static constexpr int L2 = L1 ? L / L1 : 0;
  static constexpr int NT = 256;
  static constexpr int NW = 4;
  static constexpr int W = L < 32 ? L : 32;
  static constexpr int NYB = (L + W - 1) / W;
  static constexpr size_t slab = (size_t)(N + 1) * N * sizeof(C) + (size_t)L * sizeof(C);
  static constexpr size_t line = (size_t)((L2 * (L1 + 1)) | 1) * sizeof(C);
  static constexpr int QA = L1 ? choose_q(slab, line + 2 * N * sizeof(R)) : 0;
  static constexpr int QC = L1 ? choose_q(slab, line) : 0;
  static constexpr bool ok = L1 != 0 && QA >= 1 && QC >= 1;
  static constexpr size_t smem_a = slab + QA * line + 2 * QA * N * sizeof(R);
  static constexpr size_t smem_b = (size_t)L * sizeof(C) + (size_t)L * W * sizeof(C);
  static constexpr size_t smem_c = slab + QC * line;

  static cudaError_t setup() {
    if constexpr (ok) {
      cudaError_t e;
      e = cudaFuncSetAttribute(k_fwd_xy<R, N, NT, QA>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)smem_a);
      if (e != cudaSuccess) return e;
      e = cudaFuncSetAttribute(k_zconv<R, N, NW, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)smem_b);
      if (e != cudaSuccess) return e;
      e = cudaFuncSetAttribute(k_zconv<R, N, NW, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)smem_b);
      if (e != cudaSuccess) return e;
      return cudaFuncSetAttribute(k_inv_yx<R, N, NT, QC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem_c);
    }
    return cudaErrorNotSupported;
  }
  static void fwd_xy(const void* psi, const int4* pairs, int npair, void* X2, const void* tw,
                     long long n3, cudaStream_t st) {
    if constexpr (ok)
      k_fwd_xy<R, N, NT, QA><<<dim3(N, npair), NT, smem_a, st>>>(
          static_cast<const R*>(psi), pairs, static_cast<C*>(X2), static_cast<const C*>(tw), n3);
  }
  static void zconv(void* X, const void* Gs, const void* tw, double* epart, int npair,
                    bool energy_only, cudaStream_t st) {
    if constexpr (ok) {
      const dim3 grid(NYB, N + 1, npair);
      if (energy_only)
        k_zconv<R, N, NW, true><<<grid, 32 * NW, smem_b, st>>>(
            static_cast<C*>(X), static_cast<const R*>(Gs), static_cast<const C*>(tw), epart);
      else
        k_zconv<R, N, NW, false><<<grid, 32 * NW, smem_b, st>>>(
            static_cast<C*>(X), static_cast<const R*>(Gs), static_cast<const C*>(tw), epart);
    }
  }
  static void inv_yx(const void* X3, void* V, const void* tw, int npair, cudaStream_t st) {
    if constexpr (ok)
      k_inv_yx<R, N, NT, QC><<<dim3(N, npair), NT, smem_c, st>>>(
          static_cast<const C*>(X3), static_cast<R*>(V), static_cast<const C*>(tw));
  }
  static Ops make() {
    Ops o;
    o.n = N;
    o.supported = ok;
    o.nyb = NYB;
    o.nt_a = NT;
    o.nt_c = NT;
    o.nw_b = NW;
    o.smem_a = smem_a;
    o.smem_b = smem_b;
    o.smem_c = smem_c;
    o.setup = &setup;
    o.fwd_xy = &fwd_xy;
    o.zconv = &zconv;
    o.inv_yx = &inv_yx;
    return o;
  }
};

}  // namespace exx

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
