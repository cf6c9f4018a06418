// CUDA kernels of the exact-exchange pair pipeline (sm_103a).
//
// For every orbital pair (i, j) of a pair tile (arXiv 1712.07973, Sec. 2.1:
// kernel 1 co-density, kernel 2 Poisson solve, kernel 3 products):
//
//   fwd_xy  (one CTA per z-slab and pair)
//           rho = psi_i psi_j on the slab, real-to-complex FFT of length 2n
//           along x with x >= n zero, then the pruned complex FFT of length
//           2n along y (y >= n zero).  Writes X[pair][kx][z][ky].
//   zconv   (one CTA per 32 columns (kx, ky) and pair)
//           along z: pruned forward FFT (z >= n zero), multiply by the real
//           kernel spectrum Ghat (Sec. 2.1.2; scaled by 1/(2n)^3), Parseval
//           energy sum w(kx) Ghat |rho_hat|^2, inverse FFT keeping z < n.
//           In place on X.  The kernel table slice of a CTA arrives by TMA.
//   inv_yx  (one CTA per z-slab and pair)
//           inverse FFT along y keeping y < n, complex-to-real FFT along x
//           keeping x < n: V_ij on the n^3 mesh.
//   accum   (grid-stride over mesh points, one pair tile)
//           (Vx psi)_i += -alpha f_j V_ij psi_j and, for i != j,
//           (Vx psi)_j += -alpha f_i V_ij psi_i (Eq. daction); FP32 sums
//           over the tile, FP64 accumulation across tiles, deterministic.
//
// Layouts: psi[o][z][y][x]; X[p][kx][z][ky] complex; V[p][z][y][x].
// With periodic boundary conditions (template flag PER) the grid has 2n points
// per axis, the lines are not padded and no transform is pruned; large slabs
// are split over clusters of CL = 2 or 4 CTAs.  Mixed boundary conditions give
// zconv a z line of its own (NZ, PERZ): slab = periodic x, y with a free z;
// wire = free x, y with a periodic z.
#pragma once

#include <cooperative_groups.h>
#include <cuda.h>  // CUtensorMap

#include "exx_fft.cuh"

namespace exx {

// Split of the x axis: a real line of length 2n is transformed as a complex
// line of length n (even samples + i odd samples), n = LX1 * LX2.  LX1 is even
// when n is even, so that the half of the input beyond the data is pruned.
__host__ __device__ constexpr int split_x(int n) {
  // n = 160: 10 x 16 rather than 8 x 20, so that the x passes of a quarter
  // slab (40 columns per CTA of 320 threads) run 640 and 400 units, two rounds
  // each, rather than 800 (three rounds) and 320 (fwd_xy -2%)
  if (n == 160) return 10;
  for (int a = 2; a <= 16; a += 2)
    if (n % a == 0 && n / a <= 20 && smooth7(a) && smooth7(n / a)) return a;
  if (n % 2 == 1 && n <= 16 && smooth7(n)) return n;
  return 0;
}

// Slab of the slab kernels: rows r = 0..n (k_x) of SP = ny + 1 complex values
// (columns y; ny = n, or n / CL per CTA of a CL-CTA cluster), row r starting
// at srow(r) = r SP + r / X1.  The extra slot every X1 rows skews the rows
// n2 X1 + k1 that the 16 lanes of an x-pass unit group touch (consecutive n2)
// onto distinct banks: the bank of (row, y) is 2 (n2 (X1 SP + 1) + k1 SP + y)
// mod 32, and X1 SP + 1 is odd.
__host__ __device__ constexpr int slab_elems(int n, int ny) {
  return (n + 1) * (ny + 1) + n / split_x(n) + 1;
}
template <int SP, int X1> __device__ __forceinline__ int srow(int r) { return r * SP + r / X1; }

// Padded scratch layout of one line in the [a][k1] form of the four-step:
// slot(a, k1) = a * (L1 + 1) + k1; the line stride is odd so that lines of
// different units land on different banks.
template <int L1, int L2> struct Scr {
  static constexpr int row = L1 + 1;
  static constexpr int line = (L2 * row) | 1;
};

// Load of data that other CTAs of the same launch may have written (COH, the
// persistent batched kernel: through L2, never a stale L1 or read-only-cache
// line); plain load otherwise.
template <bool COH, typename T> __device__ __forceinline__ T ldx(const T* p) {
  if constexpr (COH) return __ldcg(p);
  else return *p;
}

// Line transforms of the two boundary conditions: free (zero-padded line of
// length 2n, second half of the input zero, second half of the inverse output
// unneeded: pruned) or periodic (full line, nothing pruned).
template <int P, bool FULL, typename C> EXX_HD void dft_fwd_in(C* v) {
  if constexpr (FULL) dft<P, 1, -1>(v);
  else dft_halfin<P, -1>(v);
}
template <int P, bool FULL, typename C> EXX_HD void dft_inv_out(C* v) {
  if constexpr (FULL) dft<P, 1, 1>(v);
  else dft_halfout<P, 1>(v);
}

// Tensor-memory-access (TMA) load with an mbarrier (PTX, sm_90 and later).
__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
  // make the initialisation visible to the asynchronous (TMA) proxy
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
// 3-D tiled load of the box at coordinates (c0, c1, c2) (c0 innermost) of the
// tensor map into shared memory; completion is counted on bar in bytes.
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int c0, int c1,
                                            int c2, unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];\n" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<unsigned long long>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
      : "memory");
}
// Wait for the completion of phase `parity` of bar, polling at most `limit`
// times; false when the limit ran out.
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity, int limit) {
  for (int i = 0; i < limit; ++i) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}
constexpr int kWaitPolls = 1 << 16;  // bound of every device-side wait (a copy takes ~1 us)

// byte offset of zconv's staged kernel-table slice: after the twiddles and the
// column buffer, rounded up to 128 bytes
__host__ __device__ constexpr size_t zconv_gsm_offset(int L, int W, size_t cs) {
  return ((size_t)(L + L * W) * cs + 127) / 128 * 128;
}

// Kernel table of zconv (built by build_kernel_table): Gt[kx][kz][ky],
// kx <= n, kz, ky < 2n, the scaled kernel spectrum divided by the energy
// gains |dx(kx)|^2 |dy(ky)|^2 |dz(kz)|^2 of the FP32 forward transforms (1 in
// FP64).  Stored unfolded (Ghat is even in ky and kz) so that the gains,
// which are not, are divided out in the table itself.  For large grids
// (FOLDY) the table keeps ky folded, Gt[kx][kz][min(ky, 2n - ky)] without the
// y gain, which follows as cy[ky] = 1 / |dy(ky)|^2 (double, at
// ktab_cy_offset) and is applied to each column's energy: half the size,
// for L2 residency.
__host__ __device__ constexpr size_t ktab_cy_offset(int n, size_t rs) {
  return ((size_t)(n + 1) * (2 * n) * (n + 1) * rs + 7) / 8 * 8;
}

// One step of the split of the complex length-n spectrum Z of the (even, odd)
// sample pairs into the Hermitian half spectrum X of the real length-2n line:
// for zk = Z[k], zm = Z[n-k] (0 < k, 2k != n) and w = omega_2n^k,
// X[k] = E + w O and X[n-k] = conj(E - w O), E = (zk + conj zm) / 2,
// O = (zk - conj zm) / (2i).
template <typename C> EXX_HD void split_step(C zk, C zm, C w, C& xk, C& xm) {
  using R = typename creal<C>::type;
  const C e = mkc<C>(R(0.5) * (zk.x + zm.x), R(0.5) * (zk.y - zm.y));
  const C o = mkc<C>(R(0.5) * (zk.y + zm.y), R(-0.5) * (zk.x - zm.x));
  const C t = cmul(o, w);
  xk = cadd(e, t);
  xm = mkc<C>(e.x - t.x, t.y - e.y);
}

// ------------------------------------------------------------------ fwd_xy
// One CTA per (z-slab, pair).  Shared memory holds the slab Sl[k][y] (rows
// at srow(k), see slab_elems).  x: the complex length-n FFT of z[m] = rho[2m] + i
// rho[2m+1] runs in place in column y of Sl, followed by the split into the
// Hermitian half spectrum X[k], k = 0..n (row n is the Nyquist row).  y: the
// pruned length-2n FFT per kx row, written to HBM as X[p][kx][z][ky].  Q = 0:
// warp-owned y passes (two rows per warp); Q > 0: CTA-wide batches of Q rows.
// CL = 2 or 4 (large grids): a cluster of CL CTAs per (z-slab, pair), CTA c
// holding the columns y in [c n/CL, (c+1) n/CL) of every row; the x passes stay
// local, the y passes of a CTA's rows read the other parts of each row from the
// peers' shared memory (distributed shared memory).
// PER: periodic boundary conditions: the grid has G = 2n points per axis, the
// lines are not padded and nothing is pruned (N is then half the grid).
// fwd_xy_unit: the work of one CTA, bx = z-slab * CL + cluster rank, p = pair
// slot; k_fwd_xy launches one per block, the persistent batched kernel takes
// them from its work queue.
template <typename R, int N, int NT, int Q, int CL, bool PER>
__device__ __forceinline__ void fwd_xy_unit(const R* __restrict__ psi0,
                                            const R* const* __restrict__ psi_tab,
                                            const int4* __restrict__ pairs,
                                            cplx<R>* __restrict__ X,
                                            const cplx<R>* __restrict__ tw_g, long long n3,
                                            const int bx, const int p) {
  using C = cplx<R>;
  constexpr int L = 2 * N, L1 = split_l1(L), L2 = L / L1, H1 = L1 / 2;
  constexpr int X1 = split_x(N), X2 = N / X1;
  constexpr int G = PER ? 2 * N : N;  // grid points per axis
  constexpr bool PX = !PER && (N % 2) == 0;  // pruned x input
  constexpr int XIN = PX ? X1 / 2 : X1;
  constexpr int NIN = PER ? L1 : H1;  // nonzero inputs of the y pass-1 DFTs
  constexpr int NY = G / CL, SP = NY + 1;
  constexpr int NB = CL == 1 ? L1 : NY / L2;  // y = L2 n1 + n2 lies in half n1 / NB
  static_assert(CL == 1 || (Q == 0 && G % CL == 0 && NY % L2 == 0), "cluster split");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // twiddle tables (packed layout of build_twiddles): TY[k1][n2] = w^(n2 k1)
  // for the y pass and TX[k1][n2] = w^(2 n2 k1) for the x pass, so that
  // consecutive lanes (consecutive n2) read consecutive entries
  C* ty = reinterpret_cast<C*>(smem_raw);
  C* tx = ty + L;
  C* Sl = tx + N;  // slab, rows srow(r)

  const int tid = threadIdx.x;
  const int z = bx / CL, c = bx % CL;  // c: rank in the cluster
  const int y0 = c * NY;
  const int4 pr = pairs[p];  // (i, j, pair id, molecule slot)
  const R* psi = psi_tab ? psi_tab[pr.w] : psi0;
  const R* __restrict__ pi = psi + (long long)pr.x * n3 + (long long)z * G * G;
  const R* __restrict__ pj = psi + (long long)pr.y * n3 + (long long)z * G * G;
  for (int t = tid; t < L + N; t += NT) ty[t] = tw_g[L + t];
  __syncthreads();

  // x, pass 1: units (y, n2), n2 fastest (coalesced reads of row y); slab
  // column y - y0
  for (int u = tid; u < NY * X2; u += NT) {
    const int yl = u / X2, n2 = u - yl * X2;
    const R* ri = pi + (y0 + yl) * G;
    const R* rj = pj + (y0 + yl) * G;
    C v[X1];
#pragma unroll
    for (int n1 = 0; n1 < XIN; ++n1) {
      const int m = X2 * n1 + n2;
      const R a = (2 * m < G) ? ri[2 * m] * rj[2 * m] : R(0);
      const R b = (2 * m + 1 < G) ? ri[2 * m + 1] * rj[2 * m + 1] : R(0);
      v[n1] = mkc<C>(a, b);
    }
    if constexpr (PX) {
      dft_halfin<X1, -1>(v);
    } else {
#pragma unroll
      for (int n1 = XIN; n1 < X1; ++n1) v[n1] = mkc<C>(R(0), R(0));
      dft<X1, 1, -1>(v);
    }
    C* col = Sl + srow<SP, X1>(n2 * X1) + yl;  // rows n2 X1 + k1 at col[k1 SP]
    col[0] = v[0];
#pragma unroll
    for (int k1 = 1; k1 < X1; ++k1)  // omega_n^{n2 k1} = omega_2n^{2 n2 k1}
      col[k1 * SP] = cmul(v[k1], tx[k1 * X2 + n2]);
  }
  __syncthreads();
  // x, pass 2: units (y, k1), y fastest; in place, natural order Z[k] at row k
  for (int u = tid; u < NY * X1; u += NT) {
    const int k1 = u / NY, y = u - k1 * NY;
    C v[X2];
#pragma unroll
    for (int n2 = 0; n2 < X2; ++n2) v[n2] = Sl[srow<SP, X1>(n2 * X1 + k1) + y];
    dft<X2, 1, -1>(v);
#pragma unroll
    for (int k2 = 0; k2 < X2; ++k2) Sl[srow<SP, X1>(k1 + X1 * k2) + y] = v[k2];
  }
  __syncthreads();
  // split: X[k] = E[k] + w^k O[k], X[n-k] = conj(E[k] - w^k O[k]), with
  // E = (Z[k] + conj Z[n-k]) / 2, O = (Z[k] - conj Z[n-k]) / (2i), w = omega_2n
  // Q = 0: the two real rows kx = 0 and kx = n travel as one complex row
  // X[0] + i X[n] through the y pass (MERGE), which splits them again
  constexpr bool MERGE = Q == 0;
  for (int u = tid; u < NY * (N / 2 + 1); u += NT) {
    const int k = u / NY, y = u - k * NY;
    if (k == 0) {
      const C z0 = Sl[y];
      if constexpr (MERGE) {
        Sl[y] = mkc<C>(z0.x + z0.y, z0.x - z0.y);
      } else {
        Sl[y] = mkc<C>(z0.x + z0.y, R(0));
        Sl[srow<SP, X1>(N) + y] = mkc<C>(z0.x - z0.y, R(0));
      }
    } else if (2 * k == N) {
      const C zk = Sl[srow<SP, X1>(k) + y];
      Sl[srow<SP, X1>(k) + y] = mkc<C>(zk.x, -zk.y);
    } else {
      C xk, xm;
      C* rk = Sl + srow<SP, X1>(k) + y;
      C* rm = Sl + srow<SP, X1>(N - k) + y;
      split_step(*rk, *rm, __ldg(tw_g + k), xk, xm);  // uniform k
      *rk = xk;
      *rm = xm;
    }
  }
  // the CL parts of each row (columns [q n/CL, (q+1) n/CL) in CTA q of the
  // cluster): this CTA's slab and its peers'
  const C* hp[CL];
  if constexpr (CL > 1) {
    cooperative_groups::cluster_group cl = cooperative_groups::this_cluster();
#pragma unroll
    for (int q = 0; q < CL; ++q) hp[q] = q == c ? Sl : cl.map_shared_rank(Sl, q);
    cl.sync();  // every part transformed along x
  } else {
    hp[0] = Sl;
    __syncthreads();
  }
  // y: pruned length-2n FFT per kx row; pass 1 (DFT_L1 over n1 < L1/2, then
  // the twiddle) into a row scratch in the padded [n2][k1] layout, pass 2
  // (DFT_L2 over n2) straight to HBM
  C* S = Sl + slab_elems(N, NY);
  if constexpr (Q == 0) {
    // warp-owned: each warp transforms two kx rows at a time (one per half
    // warp) in its own scratch, synchronising with __syncwarp only; the rows
    // go round-robin over the warps of the cluster
    constexpr int NWP = NT / 32;
    const int lane = tid & 31, hr = lane >> 4, cl16 = lane & 15;
    C* Sw = S + ((tid >> 5) * 2 + hr) * Scr<L1, L2>::line;
    // a lane's first pass-1 unit is n2 = cl16 in every row it transforms: in
    // FP32 its twiddles stay in registers (FP64 lacks the registers)
    constexpr bool TWR = sizeof(R) == 4;
    C twr[TWR ? L1 : 1];
    if constexpr (TWR) {
#pragma unroll
      for (int k1 = 1; k1 < L1; ++k1) twr[k1] = cl16 < L2 ? ty[k1 * L2 + cl16] : mkc<C>(R(0), R(0));
    }
    // rows kx < n (row 0 carries rows 0 and n): 2n/(two rows per warp) rounds
    for (int r0 = 2 * (c * NWP + (tid >> 5)); r0 < N; r0 += 2 * NWP * CL) {
      const int kx = r0 + hr;
      const bool rv = kx < N;
      const int rb = srow<SP, X1>(kx);
      if (rv && cl16 < L2) {
        C v[L1];
#pragma unroll
        for (int n1 = 0; n1 < NIN; ++n1) v[n1] = hp[n1 / NB][rb + L2 * (n1 % NB) + cl16];
        dft_fwd_in<L1, PER>(v);
        C* o = Sw + cl16 * Scr<L1, L2>::row;
        o[0] = v[0];
#pragma unroll
        for (int k1 = 1; k1 < L1; ++k1) o[k1] = cmul(v[k1], TWR ? twr[TWR ? k1 : 0] : ty[k1 * L2 + cl16]);
      }
      if constexpr (!PER && L2 > 16 && L2 <= 24) {
        // L2 > 16 (n = 160): the units n2 = 16 .. L2-1 as half units, lanes 2u
        // and 2u + 1 of the half warp taking the even and odd outputs of unit
        // 16 + u (the two length-L1/2 DFTs of the pruned transform), so that
        // the second round costs half a unit (fwd_xy -5% at 160^3); the same
        // operations as dft_halfin, so the same results
        if (rv && cl16 < 2 * (L2 - 16)) {
          const int n2 = 16 + (cl16 >> 1), hh = cl16 & 1;
          C e[H1];
#pragma unroll
          for (int n1 = 0; n1 < H1; ++n1) e[n1] = hp[n1 / NB][rb + L2 * (n1 % NB) + n2];
          if (hh) sfor<H1>([&](auto J) { e[J] = twmul<-1, L1, (int)J>(e[J]); });
          dft<H1, 1, -1>(e);
          C* o = Sw + n2 * Scr<L1, L2>::row;
#pragma unroll
          for (int k = 0; k < H1; ++k) {
            const int k1 = 2 * k + hh;
            o[k1] = k1 == 0 ? e[0] : cmul(e[k], ty[k1 * L2 + n2]);
          }
        }
      } else {
        for (int n2 = cl16 + 16; n2 < L2; n2 += 16) {  // L2 > 16: further units
          if (rv) {
            C v[L1];
#pragma unroll
            for (int n1 = 0; n1 < NIN; ++n1) v[n1] = hp[n1 / NB][rb + L2 * (n1 % NB) + n2];
            dft_fwd_in<L1, PER>(v);
            C* o = Sw + n2 * Scr<L1, L2>::row;
            o[0] = v[0];
#pragma unroll
            for (int k1 = 1; k1 < L1; ++k1) o[k1] = cmul(v[k1], ty[k1 * L2 + n2]);
          }
        }
      }
      __syncwarp();
      if (rv && cl16 < L1) {
        const C* q = Sw + cl16;
        C v[L2];
#pragma unroll
        for (int n2 = 0; n2 < L2; ++n2) v[n2] = q[n2 * Scr<L1, L2>::row];
        dft<L2, 1, -1>(v);
        C* out = X + (((long long)p * (N + 1) + kx) * G + z) * L + cl16;
        if (kx == 0) {
          // split C = Y0 + i YN (Y0, YN spectra of real rows):
          // Y0[k] = (C[k] + conj C[-k]) / 2, YN[k] = (C[k] - conj C[-k]) / (2i).
          // C[k1 + L1 k2] is v[k2] of lane k1; C[-k] is v[(L2 - k2) % L2] of
          // lane 0 for k1 = 0, else v[L2 - 1 - k2] of lane L1 - k1.
          const unsigned mask = (1u << L1) - 1u;  // lanes 0..L1-1 of half warp 0
          const int partner = (L1 - cl16) % L1;
          C* outN = X + (((long long)p * (N + 1) + N) * G + z) * L + cl16;
#pragma unroll
          for (int k2 = 0; k2 < L2; ++k2) {
            C b;
            b.x = __shfl_sync(mask, v[L2 - 1 - k2].x, partner, 16);
            b.y = __shfl_sync(mask, v[L2 - 1 - k2].y, partner, 16);
            if (cl16 == 0) b = v[(L2 - k2) % L2];
            const C a = v[k2];
            out[L1 * k2] = mkc<C>(R(0.5) * (a.x + b.x), R(0.5) * (a.y - b.y));
            outN[L1 * k2] = mkc<C>(R(0.5) * (a.y + b.y), R(0.5) * (b.x - a.x));
          }
        } else {
#pragma unroll
          for (int k2 = 0; k2 < L2; ++k2) out[L1 * k2] = v[k2];
        }
      }
      __syncwarp();
    }
    // the peers may still be reading this CTA's part
    if constexpr (CL > 1) cooperative_groups::this_cluster().sync();
  } else {
    // CTA-wide batches of Q rows
    for (int r0 = 0; r0 <= N; r0 += Q) {
      const int nr = min(Q, N + 1 - r0);
      // units (kx row, n2) with the row fastest: the slab reads stride SP and
      // the scratch writes stride the (odd) line length, both bank-conflict free
      for (int u = tid; u < nr * L2; u += NT) {
        const int n2 = u / nr, r = u - n2 * nr;
        const C* row = Sl + srow<SP, X1>(r0 + r);
        C v[L1];
#pragma unroll
        for (int n1 = 0; n1 < NIN; ++n1) v[n1] = row[L2 * n1 + n2];
        dft_fwd_in<L1, PER>(v);
        C* o = S + r * Scr<L1, L2>::line + n2 * Scr<L1, L2>::row;
        o[0] = v[0];
#pragma unroll
        for (int k1 = 1; k1 < L1; ++k1) o[k1] = cmul(v[k1], ty[k1 * L2 + n2]);
      }
      __syncthreads();
      for (int u = tid; u < nr * L1; u += NT) {
        const int r = u / L1, k1 = u - r * L1;
        const C* q = S + r * Scr<L1, L2>::line + k1;
        C v[L2];
#pragma unroll
        for (int n2 = 0; n2 < L2; ++n2) v[n2] = q[n2 * Scr<L1, L2>::row];
        dft<L2, 1, -1>(v);
        C* out = X + (((long long)p * (N + 1) + (r0 + r)) * G + z) * L + k1;
#pragma unroll
        for (int k2 = 0; k2 < L2; ++k2) out[L1 * k2] = v[k2];
      }
      __syncthreads();
    }
  }
}

template <typename R, int N, int NT, int MINB, int Q, int CL, bool PER>
__global__ void __launch_bounds__(NT, MINB)
k_fwd_xy(const R* __restrict__ psi0, const R* const* __restrict__ psi_tab,
         const int4* __restrict__ pairs, cplx<R>* __restrict__ X, const cplx<R>* __restrict__ tw_g,
         long long n3) {
  // grid (CL * pairs, z): the CTAs of one z-slab for all pairs of the tile run
  // together, so the tile's orbital planes at that z are read from L2 once
  // they are in (at 160^3 the tile's orbitals, 262 MB, exceed L2)
  fwd_xy_unit<R, N, NT, Q, CL, PER>(psi0, psi_tab, pairs, X, tw_g, n3,
                                    blockIdx.y * CL + blockIdx.x % CL, blockIdx.x / CL);
}

// ------------------------------------------------------------------- zconv
// One CTA per (32 consecutive ky columns, kx, pair); lane = column, warps
// share the sub-DFTs of each pass.  Along z: pruned forward FFT (pass 1 of
// length L1 over z = L2 n1 + n2, pass 2 of length L2), multiply by the kernel
// table (Ghat/(2n)^3) with the Parseval energy w(kx) Ghat |rho_hat|^2, inverse
// FFT keeping z < n.  In place on X.  STAGE: the CTA's slice of the kernel
// table, Gt[kx][kz][ky0 .. ky0 + W), is brought into shared memory by one TMA
// load (tensor map gmap, box W x 2n x 1) that overlaps the first pass (FP32,
// and only where it costs no occupancy); otherwise the values are read from
// global memory in the second pass.  A wait that runs out sets err[0];
// err[1] != 0 (a test hook set by the host) skips issuing the copy, so that
// the bounded wait runs out on purpose.
// (N, PER) describe the x and y axes (kx <= N, ky < 2N), (NZ, PERZ) the z
// transform (length 2NZ, tw_g its twiddles); they differ for the mixed
// boundary conditions: slab (x, y periodic, z free) and wire (x, y free,
// z periodic).
// zconv_unit: the work of one CTA (yb = column block, kx, p = pair slot).
template <typename R, int N, int NW, int MINB, bool STAGE, bool FOLDY, bool PER, bool ENERGY_ONLY,
          int NZ, bool PERZ, bool COH>
__device__ __forceinline__ void zconv_unit(cplx<R>* __restrict__ X, const R* __restrict__ Gs,
                                           const cplx<R>* __restrict__ tw_g,
                                           double* __restrict__ epart, const CUtensorMap* gmap,
                                           int* __restrict__ err, const int yb, const int kx,
                                           const int p) {
  using C = cplx<R>;
  constexpr int LY = 2 * N;  // ky extent: the row stride of X and of the kernel table
  constexpr int L = 2 * NZ, L1 = split_z(L), L2 = L / L1, H1 = L1 / 2;
  constexpr int W = LY < 32 ? LY : 32;
  constexpr int M = N + 1;
  static_assert((PER ? 2 * N : N) == (PERZ ? 2 * NZ : NZ), "one grid size on all axes");
  static_assert(!FOLDY || (NZ == N && PERZ == PER), "folded tables are cubic");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* tw = reinterpret_cast<C*>(smem_raw);  // w^k [L]
  C* buf = tw + L;                         // [L slots][W]
  // [L][W] (STAGE): the TMA destination, 128-byte aligned in the shared window
  // (the dynamic allocation starts after the static variables, so the base is
  // aligned at run time; the allocation has 128 bytes of slack for this)
  R* gsm = reinterpret_cast<R*>(smem_raw + zconv_gsm_offset(L, W, sizeof(C)) +
                                ((128u - (smem_u32(smem_raw) & 127u)) & 127u));
  __shared__ double red[NW];
  __shared__ __align__(8) unsigned long long gbar;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int NYB = (LY + W - 1) / W;  // column blocks per kx plane
  const int ky = yb * W + lane;
  const bool valid = lane < W && ky < LY;
  if constexpr (STAGE) {
    static_assert(sizeof(R) == 4 && (W * sizeof(R)) % 16 == 0 && L <= 256, "TMA box");
    if (tid == 0) {  // out-of-range ky of a partial last block read as zero
      mbar_init(&gbar, 1);
      if (err[1] != 0) {
        // test hook: no copy, nothing arrives, the wait below runs out
      } else if ((smem_u32(gsm) & 127u) == 0) {
        mbar_expect_tx(&gbar, (unsigned)(L * W * sizeof(R)));
        tma_load_3d(gsm, gmap, yb * W, 0, kx, &gbar);
      } else {  // never expected: report instead of issuing an unaligned copy
        atomicExch(err, 2);
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(&gbar)) : "memory");
      }
    }
  }
  for (int t = tid; t < L; t += 32 * NW) tw[t] = tw_g[t];
  constexpr int GR = FOLDY ? N + 1 : LY;  // table row length
  const int kyt = FOLDY ? (ky <= N ? ky : LY - ky) : ky;
  const R* __restrict__ Gk = Gs + (long long)kx * L * GR + (valid ? kyt : 0);
  double cyl = 1.0;
  if constexpr (FOLDY) {
    static_assert(!STAGE, "staging reads unfolded rows");
    if (valid)
      cyl = reinterpret_cast<const double*>(reinterpret_cast<const unsigned char*>(Gs) +
                                            ktab_cy_offset(N, sizeof(R)))[ky];
  }
  constexpr int G = PERZ ? 2 * NZ : NZ;  // z planes stored (grid points per axis)
  constexpr int NIN = PERZ ? L1 : H1;    // nonzero inputs / kept outputs per DFT_L1
  C* col = X + (((long long)p * M + kx) * G) * LY + (valid ? ky : 0);
  {
    // the CTA's whole column block (G rows of W columns) is requested into L2
    // first, so that the warps' second pass-1 units find their rows there
    // (-4% zconv at 160^3; requesting the block of the CTA one wave ahead
    // instead measured slower)
    constexpr int PL = 128 / (int)sizeof(C), LPR = (W + PL - 1) / PL;  // lines per z row
    const C* blk = X + (((long long)p * M + kx) * G) * LY + yb * W;
    const int wr = min(W, LY - yb * W);  // columns of this block
    for (int t = tid; t < G * LPR; t += 32 * NW)
      if ((t % LPR) * PL < wr)
        asm volatile("prefetch.global.L2 [%0];\n" ::"l"(blk + (long long)(t / LPR) * LY + (t % LPR) * PL));
  }
  __syncthreads();

  // forward, pass 1
  for (int n2 = warp; n2 < L2; n2 += NW) {
    C v[L1];
#pragma unroll
    for (int n1 = 0; n1 < NIN; ++n1)
      v[n1] = valid ? ldx<COH>(col + (long long)(L2 * n1 + n2) * LY) : mkc<C>(R(0), R(0));
    dft_fwd_in<L1, PERZ>(v);
    if (lane < W) {
      buf[(n2 * L1) * W + lane] = v[0];
#pragma unroll
      for (int k1 = 1; k1 < L1; ++k1)
        buf[(n2 * L1 + k1) * W + lane] = cmul(v[k1], tw[n2 * k1]);
    }
  }
  if constexpr (STAGE) {
    if (!mbar_wait(&gbar, 0, kWaitPolls)) atomicExch(err, 1);
  }
  __syncthreads();

  // forward pass 2, kernel multiply, energy, inverse pass 1
  double eacc = 0.0;
  // PF (unstaged, with the register budget of two CTAs per SM): the unit's
  // kernel-table values are requested before its transform
  constexpr bool PF = !STAGE && sizeof(R) == 4 && 65536 / (32 * NW * MINB) >= 96;
  for (int k1 = warp; k1 < L1; k1 += NW) {
    R gp[PF ? L2 : 1];
    if constexpr (PF) {
#pragma unroll
      for (int k2 = 0; k2 < L2; ++k2) gp[k2] = valid ? __ldg(Gk + (k1 + L1 * k2) * GR) : R(0);
    }
    C v[L2];
#pragma unroll
    for (int n2 = 0; n2 < L2; ++n2)
      v[n2] = lane < W ? buf[(n2 * L1 + k1) * W + lane] : mkc<C>(R(0), R(0));
    dft<L2, 1, -1>(v);
    R es = R(0);
#pragma unroll
    for (int k2 = 0; k2 < L2; ++k2) {
      const int kz = k1 + L1 * k2;
      R gv;
      if constexpr (STAGE) gv = valid ? gsm[kz * W + lane] : R(0);  // lane < W
      else if constexpr (PF) gv = gp[k2];
      else gv = valid ? __ldg(Gk + kz * GR) : R(0);
      // (the squares are independent of es: one dependent add per value;
      // accumulating (Ghat x) x + (Ghat y) y into es measured 2.6% slower)
      es += gv * (v[k2].x * v[k2].x + v[k2].y * v[k2].y);
      v[k2] = cscale(v[k2], gv);
    }
    eacc += (double)es;
    if constexpr (!ENERGY_ONLY) {
      dft<L2, 1, 1>(v);
      if (lane < W) {
        buf[k1 * W + lane] = v[0];
#pragma unroll
        for (int m2 = 1; m2 < L2; ++m2) buf[(m2 * L1 + k1) * W + lane] = cmulc(v[m2], tw[m2 * k1]);
      }
    }
  }
  if constexpr (!ENERGY_ONLY) {
    __syncthreads();
    // inverse, pass 2: only z = L2 m1 + m2 < n is kept
    for (int m2 = warp; m2 < L2; m2 += NW) {
      C v[L1];
#pragma unroll
      for (int k1 = 0; k1 < L1; ++k1)
        v[k1] = lane < W ? buf[(m2 * L1 + k1) * W + lane] : mkc<C>(R(0), R(0));
      dft_inv_out<L1, PERZ>(v);
      if (valid) {
#pragma unroll
        for (int m1 = 0; m1 < NIN; ++m1) col[(long long)(L2 * m1 + m2) * LY] = v[m1];
      }
    }
  }
  // Parseval energy of this block (fixed-order reduction)
  if constexpr (FOLDY) eacc *= cyl;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) eacc += __shfl_xor_sync(0xffffffffu, eacc, o);
  if (lane == 0) red[warp] = eacc;
  __syncthreads();
  if (tid == 0) {
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < NW; ++w) s += red[w];
    const double wk = (kx == 0 || kx == N) ? 1.0 : 2.0;
    epart[((long long)p * M + kx) * NYB + yb] = wk * s;
  }
}

template <typename R, int N, int NW, int MINB, bool STAGE, bool FOLDY, bool PER, bool ENERGY_ONLY,
          int NZ = N, bool PERZ = PER>
__global__ void __launch_bounds__(32 * NW, MINB)
k_zconv(cplx<R>* __restrict__ X, const R* __restrict__ Gs, const cplx<R>* __restrict__ tw_g,
        double* __restrict__ epart, const __grid_constant__ CUtensorMap gmap, int* __restrict__ err) {
  // grid (column blocks, pairs, kx): consecutive CTAs read adjacent columns of
  // the same rows of one pair's spectrum, and the CTAs of one kx plane for all
  // pairs of the tile run together, so the plane's kernel-table rows come from
  // L2 for every pair
  zconv_unit<R, N, NW, MINB, STAGE, FOLDY, PER, ENERGY_ONLY, NZ, PERZ, false>(
      X, Gs, tw_g, epart, &gmap, err, blockIdx.x, blockIdx.z, blockIdx.y);
}

// ------------------------------------------------------------------ inv_yx
// Request row kx of pair slot p at plane z of the spectrum X[p][kx][z][ky]
// into L2 (nothing for kx >= n): lane l < 16 of a half warp touches the row's
// 128-byte lines l, l + 16, ... (whole lines only: every address lies in the
// row).
template <int N, int G, typename C>
__device__ __forceinline__ void prefetch_row_l2(const C* X, int p, int kx, int z, int l) {
  constexpr int L = 2 * N, PL = 128 / (int)sizeof(C);
  if (kx >= N) return;
  const C* row = X + (((long long)p * (N + 1) + kx) * G + z) * L;
  for (int ln = l; ln < L / PL; ln += 16)
    asm volatile("prefetch.global.L2 [%0];\n" ::"l"(row + ln * PL));
}

// One CTA per (z-slab, pair).  y: inverse FFT of each kx row (pruned output
// y < n) from HBM into the slab Sl[kx][y]; x: the Hermitian half
// spectrum of each line is folded into a complex length-n spectrum
// Z[k] = E'[k] + i O'[k] (E' = X[k] + conj X[n-k], O' = (X[k] - conj X[n-k])
// w^-k), whose inverse FFT (in place in column y) gives the even and odd
// samples of the real line: V[2m] = Re, V[2m+1] = Im, kept for x < n.
// CL = 2 or 4: CTA cluster as in fwd_xy; a CTA's y passes write the other
// parts of each row into the peers' slabs, then each CTA transforms its own
// columns.
// PER: periodic boundary conditions (see fwd_xy).
// inv_yx_unit: the work of one CTA (bx = z-slab * CL + cluster rank, p = pair).
template <typename R, int N, int NT, int Q, int CL, bool PER, bool COH>
__device__ __forceinline__ void inv_yx_unit(const cplx<R>* __restrict__ X, R* __restrict__ V,
                                            const cplx<R>* __restrict__ tw_g, const int bx,
                                            const int p) {
  using C = cplx<R>;
  constexpr int L = 2 * N, L1 = split_l1(L), L2 = L / L1, H1 = L1 / 2;
  constexpr int X1 = split_x(N), X2 = N / X1;
  constexpr int G = PER ? 2 * N : N;  // grid points per axis
  constexpr bool PX = !PER && (N % 2) == 0;
  constexpr int XOUT = PX ? X1 / 2 : X1;
  constexpr int NOUT = PER ? L1 : H1;  // kept outputs of the y pass-2 DFTs
  constexpr int NY = G / CL, SP = NY + 1;
  constexpr int NB = CL == 1 ? L1 : NY / L2;  // y = L2 m1 + m2 lies in half m1 / NB
  static_assert(CL == 1 || (Q == 0 && G % CL == 0 && NY % L2 == 0), "cluster split");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* tw = reinterpret_cast<C*>(smem_raw);  // w^k, high parts [L]
  C* ti = tw + L;                          // TI[m2][k1] = w^(m2 k1) [L] (see fwd_xy)
  C* Sl = ti + L;                          // slab, rows srow(r) (see fwd_xy)

  const int tid = threadIdx.x;
  const int z = bx / CL, c = bx % CL;  // c: rank in the cluster
  const int y0 = c * NY;
  // warp-owned y passes: the half warp's first row is requested into L2 before
  // the set-up, each later row one round ahead (in the y loop)
  if constexpr (Q == 0)
    prefetch_row_l2<N, G>(X, p, 2 * (c * (NT / 32) + (tid >> 5)) + ((tid & 31) >> 4), z, tid & 15);
  for (int t = tid; t < L; t += NT) tw[t] = tw_g[t];
  for (int t = tid; t < L; t += NT) ti[t] = tw_g[2 * L + N + t];
  C* hp[CL];  // row parts (see fwd_xy)
  if constexpr (CL > 1) {
    cooperative_groups::cluster_group cl = cooperative_groups::this_cluster();
#pragma unroll
    for (int q = 0; q < CL; ++q) hp[q] = q == c ? Sl : cl.map_shared_rank(Sl, q);
    cl.sync();  // the peers have started (their shared memory may be written)
  } else {
    hp[0] = Sl;
    __syncthreads();
  }
  // y: inverse length-2n FFT per kx row keeping y < n; pass 1 (DFT_L2 over
  // k2, twiddle) from HBM into a row scratch, pass 2 (pruned-output DFT_L1
  // over k1) into the slab
  C* S = Sl + slab_elems(N, NY);
  if constexpr (Q == 0) {
    // warp-owned: two kx rows per warp (one per half warp), own scratch; the
    // rows go round-robin over the warps of the cluster
    constexpr int NWP = NT / 32;
    const int lane = tid & 31, hr = lane >> 4, cl16 = lane & 15;
    C* Sw = S + ((tid >> 5) * 2 + hr) * Scr<L1, L2>::line;
    // a lane's pass-1 unit is k1 = cl16 in every row: in FP32 its twiddles
    // stay in registers
    constexpr bool TWR = sizeof(R) == 4;
    C twr[TWR ? L2 : 1];
    if constexpr (TWR) {
#pragma unroll
      for (int m2 = 1; m2 < L2; ++m2) twr[m2] = cl16 < L1 ? ti[m2 * L1 + cl16] : mkc<C>(R(0), R(0));
    }
    // rows kx < n; row 0 transforms X[0] + i X[n]: both give real lines
    // (Hermitian in ky), which come out as the real and imaginary parts
    for (int r0 = 2 * (c * NWP + (tid >> 5)); r0 < N; r0 += 2 * NWP * CL) {
      const int kx = r0 + hr;
      const bool rv = kx < N;
      prefetch_row_l2<N, G>(X, p, kx + 2 * NWP * CL, z, cl16);  // the next round's row
      if (rv && cl16 < L1) {
        const C* in = X + (((long long)p * (N + 1) + kx) * G + z) * L + cl16;
        C v[L2];
#pragma unroll
        for (int k2 = 0; k2 < L2; ++k2) v[k2] = ldx<COH>(in + L1 * k2);
        if (kx == 0) {
          const C* inN = X + (((long long)p * (N + 1) + N) * G + z) * L + cl16;
#pragma unroll
          for (int k2 = 0; k2 < L2; ++k2) {
            const C w = ldx<COH>(inN + L1 * k2);
            v[k2] = mkc<C>(v[k2].x - w.y, v[k2].y + w.x);
          }
        }
        dft<L2, 1, 1>(v);
        C* q = Sw + cl16;
        q[0] = v[0];
#pragma unroll
        for (int m2 = 1; m2 < L2; ++m2)
          q[m2 * Scr<L1, L2>::row] = cmulc(v[m2], TWR ? twr[TWR ? m2 : 0] : ti[m2 * L1 + cl16]);
      }
      __syncwarp();
      for (int m2 = cl16; m2 < L2; m2 += 16) {
        if (rv) {
          const C* q = Sw + m2 * Scr<L1, L2>::row;
          C v[L1];
#pragma unroll
          for (int k1 = 0; k1 < L1; ++k1) v[k1] = q[k1];
          dft_inv_out<L1, PER>(v);
          const int rb = srow<SP, X1>(kx);
#pragma unroll
          for (int m1 = 0; m1 < NOUT; ++m1) hp[m1 / NB][rb + L2 * (m1 % NB) + m2] = v[m1];
        }
      }
      __syncwarp();
    }
    if constexpr (CL > 1) cooperative_groups::this_cluster().sync();  // every part written
    else __syncthreads();
  } else {
    for (int r0 = 0; r0 <= N; r0 += Q) {
      const int nr = min(Q, N + 1 - r0);
      for (int u = tid; u < nr * L1; u += NT) {
        const int r = u / L1, k1 = u - r * L1;
        const C* in = X + (((long long)p * (N + 1) + (r0 + r)) * G + z) * L + k1;
        C v[L2];
#pragma unroll
        for (int k2 = 0; k2 < L2; ++k2) v[k2] = ldx<COH>(in + L1 * k2);
        dft<L2, 1, 1>(v);
        C* q = S + r * Scr<L1, L2>::line + k1;
        q[0] = v[0];
#pragma unroll
        for (int m2 = 1; m2 < L2; ++m2) q[m2 * Scr<L1, L2>::row] = cmulc(v[m2], ti[m2 * L1 + k1]);
      }
      __syncthreads();
      for (int u = tid; u < nr * L2; u += NT) {  // row fastest (see fwd_xy)
        const int m2 = u / nr, r = u - m2 * nr;
        const C* q = S + r * Scr<L1, L2>::line + m2 * Scr<L1, L2>::row;
        C v[L1];
#pragma unroll
        for (int k1 = 0; k1 < L1; ++k1) v[k1] = q[k1];
        dft_inv_out<L1, PER>(v);
        C* row = Sl + srow<SP, X1>(r0 + r);
#pragma unroll
        for (int m1 = 0; m1 < NOUT; ++m1) row[L2 * m1 + m2] = v[m1];
      }
      __syncthreads();
    }
  }
  // fold the half spectrum into Z (units (y, k), k = 0..n/2, y fastest);
  // Q = 0: row 0 holds the lines of rows 0 and n as (real, imaginary) parts
  constexpr bool MERGE = Q == 0;
  for (int u = tid; u < NY * (N / 2 + 1); u += NT) {
    const int k = u / NY, y = u - k * NY;
    if (k == 0) {
      const R x0 = Sl[y].x, xn = MERGE ? Sl[y].y : Sl[srow<SP, X1>(N) + y].x;
      Sl[y] = mkc<C>(x0 + xn, x0 - xn);
    } else if (2 * k == N) {
      C* rk = Sl + srow<SP, X1>(k) + y;
      const C xk = *rk;
      *rk = mkc<C>(R(2) * xk.x, R(-2) * xk.y);
    } else {
      C* rk = Sl + srow<SP, X1>(k) + y;
      C* rm = Sl + srow<SP, X1>(N - k) + y;
      const C xk = *rk, xm = *rm;
      const C e = mkc<C>(xk.x + xm.x, xk.y - xm.y);
      const C d = mkc<C>(xk.x - xm.x, xk.y + xm.y);
      const C o = cmulc(d, tw[k]);
      *rk = mkc<C>(e.x - o.y, e.y + o.x);
      *rm = mkc<C>(e.x + o.y, o.x - e.y);
    }
  }
  __syncthreads();
  // x inverse, pass 1: units (y, k1), y fastest; in place over rows k1 + X1 k2
  for (int u = tid; u < NY * X1; u += NT) {
    const int k1 = u / NY, y = u - k1 * NY;
    C v[X2];
#pragma unroll
    for (int k2 = 0; k2 < X2; ++k2) v[k2] = Sl[srow<SP, X1>(k1 + X1 * k2) + y];
    dft<X2, 1, 1>(v);
    Sl[srow<SP, X1>(k1) + y] = v[0];
#pragma unroll
    for (int m2 = 1; m2 < X2; ++m2) Sl[srow<SP, X1>(m2 * X1 + k1) + y] = cmulc(v[m2], tw[2 * m2 * k1]);
  }
  __syncthreads();
  // x inverse, pass 2: units (y, m2), m2 fastest (coalesced writes of row y)
  R* Vz = V + ((long long)p * G + z) * G * G;
  for (int u = tid; u < NY * X2; u += NT) {
    const int y = u / X2, m2 = u - y * X2;
    C v[X1];
#pragma unroll
    for (int k1 = 0; k1 < X1; ++k1) v[k1] = Sl[srow<SP, X1>(m2 * X1 + k1) + y];
    if constexpr (PX) dft_halfout<X1, 1>(v);
    else dft<X1, 1, 1>(v);
    R* row = Vz + (long long)(y0 + y) * G;
#pragma unroll
    for (int m1 = 0; m1 < XOUT; ++m1) {
      const int m = X2 * m1 + m2;
      if (2 * m < G) row[2 * m] = v[m1].x;
      if (2 * m + 1 < G) row[2 * m + 1] = v[m1].y;
    }
  }
}

template <typename R, int N, int NT, int MINB, int Q, int CL, bool PER>
__global__ void __launch_bounds__(NT, MINB)
k_inv_yx(const cplx<R>* __restrict__ X, R* __restrict__ V, const cplx<R>* __restrict__ tw_g) {
  inv_yx_unit<R, N, NT, Q, CL, PER, false>(X, V, tw_g, blockIdx.x, blockIdx.y);
}

// ------------------------------------------------------------------- accum
// One pair tile: orbitals i0..i0+ti-1 (block I) and j0..j0+tj-1 (block J);
// off-diagonal tiles hold all ti*tj pairs (slot a*tj + b), diagonal tiles
// (I == J) the ti(ti+1)/2 pairs a <= b in row-major order.  Each thread owns
// VEC consecutive mesh points (vector loads); the J loop is outermost so that
// only the I-side partial sums stay live.
template <typename R, int VEC> struct vecty;
template <> struct vecty<float, 4> { using type = float4; };
template <> struct vecty<float, 2> { using type = float2; };
template <> struct vecty<float, 1> { using type = float; };
template <> struct vecty<double, 2> { using type = double2; };
template <> struct vecty<double, 1> { using type = double; };

template <typename R, int VEC, bool COH = false>
__device__ __forceinline__ void vload(const R* p, R (&v)[VEC]) {
  if constexpr (VEC == 1) {
    v[0] = ldx<COH>(p);
  } else {
    using V = typename vecty<R, VEC>::type;
    const V t = ldx<COH>(reinterpret_cast<const V*>(p));
    const R* q = reinterpret_cast<const R*>(&t);
#pragma unroll
    for (int e = 0; e < VEC; ++e) v[e] = q[e];
  }
}
// vx[0..VEC) += c * a  (FP64)
template <typename R, int VEC, bool COH = false>
__device__ __forceinline__ void vacc(double* p, double c, const R (&a)[VEC]) {
  if constexpr (VEC == 4) {
    double2* q = reinterpret_cast<double2*>(p);
    double2 u = ldx<COH>(q), w = ldx<COH>(q + 1);
    u.x += c * (double)a[0];
    u.y += c * (double)a[1];
    w.x += c * (double)a[2];
    w.y += c * (double)a[3];
    q[0] = u;
    q[1] = w;
  } else if constexpr (VEC == 2) {
    double2* q = reinterpret_cast<double2*>(p);
    double2 u = ldx<COH>(q);
    u.x += c * (double)a[0];
    u.y += c * (double)a[1];
    q[0] = u;
  } else {
    p[0] = ldx<COH>(p) + c * (double)a[0];
  }
}

// Products and accumulation of one tile at the VEC mesh points from r.
// MODE 0: any tile; MODE 1: full off-diagonal tile (ti = tj = TM); MODE 2:
// full diagonal tile.  The full modes make every loop bound and branch a
// compile-time constant, so that all loads of a J step can be issued at once
// (with the register budget of two CTAs per SM: 4.9 -> 3.8 ms per exx_apply
// at n = 96, 64 orbitals).
// gs = 0: the exchange action, vx_k += c * sum; gs > 0: the gradient of E_x,
// vx_k += c gs f_k * sum (gs = 2 h^3: dE_x/dpsi_k = 2 f_k h^3 (Vx psi)_k,
// Eq. daction), the per-orbital factor folded into the FP64 accumulation.
template <typename R, int TM, int VEC, int MODE, bool COH = false>
__device__ __forceinline__ void accum_tile(const R* __restrict__ psi, const R* __restrict__ V,
                                           double* __restrict__ vx,
                                           const double* __restrict__ occ, int i0, int ti_,
                                           int j0, int tj_, int diag_, double c, double gs,
                                           long long n3, long long r) {
  const int ti = MODE ? TM : ti_, tj = MODE ? TM : tj_;
  const bool diag = MODE == 2 ? true : MODE == 1 ? false : diag_ != 0;
  R fi[TM];
#pragma unroll
  for (int a = 0; a < TM; ++a) fi[a] = a < ti ? (R)occ[i0 + a] : R(0);
  R pi[TM][VEC], ai[TM][VEC];
#pragma unroll
  for (int a = 0; a < TM; ++a) {
    if (a < ti) vload<R, VEC>(psi + (long long)(i0 + a) * n3 + r, pi[a]);
#pragma unroll
    for (int e = 0; e < VEC; ++e) ai[a][e] = R(0);
  }
#pragma unroll
  for (int b = 0; b < TM; ++b) {
    if (b >= tj) break;
    const R fb = (R)occ[j0 + b];
    R pb[VEC], aj[VEC];
    if (diag) {
#pragma unroll
      for (int e = 0; e < VEC; ++e) pb[e] = pi[b][e];
    } else {
      vload<R, VEC>(psi + (long long)(j0 + b) * n3 + r, pb);
    }
#pragma unroll
    for (int e = 0; e < VEC; ++e) aj[e] = R(0);
#pragma unroll
    for (int a = 0; a < TM; ++a) {
      if (a >= ti || (diag && a > b)) continue;
      const int slot = diag ? a * tj - (a * (a - 1)) / 2 + (b - a) : a * tj + b;
      R v[VEC];
      vload<R, VEC, COH>(V + (long long)slot * n3 + r, v);
#pragma unroll
      for (int e = 0; e < VEC; ++e) {
        ai[a][e] += fb * v[e] * pb[e];
        if (!(diag && a == b)) aj[e] += fi[a] * v[e] * pi[a][e];
      }
    }
    if (diag) {
      // J side of a diagonal tile is the I side: fold into ai[b]
#pragma unroll
      for (int e = 0; e < VEC; ++e) ai[b][e] += aj[e];
    } else {
      const double cb = gs != 0.0 ? c * (gs * occ[j0 + b]) : c;
      vacc<R, VEC, COH>(vx + (long long)(j0 + b) * n3 + r, cb, aj);
    }
  }
#pragma unroll
  for (int a = 0; a < TM; ++a)
    if (a < ti) {
      const double ca = gs != 0.0 ? c * (gs * occ[i0 + a]) : c;
      vacc<R, VEC, COH>(vx + (long long)(i0 + a) * n3 + r, ca, ai[a]);
    }
}

template <typename R, int TM, int VEC, int MODE>
__global__ void __launch_bounds__(256, (sizeof(R) == 4 && MODE == 0) ? 3 : 2)
k_accum(const R* __restrict__ psi, const R* __restrict__ V, double* __restrict__ vx,
        const double* __restrict__ occ, int i0, int ti, int j0, int tj, int diag, double c,
        double gs, long long n3) {
  const long long r = (blockIdx.x * (long long)blockDim.x + threadIdx.x) * VEC;
  if (r >= n3) return;
  accum_tile<R, TM, VEC, MODE>(psi, V, vx, occ, i0, ti, j0, tj, diag, c, gs, n3, r);
}

// Tile descriptor of a batched wave (tiles of different molecules, or of
// disjoint orbital blocks, so that no two touch the same accumulator).
struct TileDesc {
  int i0, ti, j0, tj, diag;
  int voff;   // first pair slot of the tile in V
  int mol;    // molecule slot: psi_tab[mol], vx_tab[mol], occ + occ_off[mol]
  int occ_off;
  double c;   // -alpha of the molecule
  double g2h3;  // 2 h^3 of the molecule (gradient calls)
};

// One tile per blockIdx.y; full tiles take the specialised bodies (the branch
// is uniform over a block).  grad != 0: gradient of E_x (see accum_tile).
template <typename R, int TM, int VEC, bool COH>
__device__ __forceinline__ void accum_batch_unit(const R* const* __restrict__ psi_tab,
                                                 const R* __restrict__ V,
                                                 double* const* __restrict__ vx_tab,
                                                 const double* __restrict__ occ,
                                                 const TileDesc* __restrict__ tiles, int grad,
                                                 long long n3, const int bx, const int by,
                                                 const int nt) {
  const TileDesc t = tiles[by];
  const long long r = (bx * (long long)nt + threadIdx.x) * VEC;
  if (r >= n3) return;
  const R* __restrict__ psi = psi_tab[t.mol];
  double* __restrict__ vx = vx_tab[t.mol];
  const double* __restrict__ oc = occ + t.occ_off;
  const R* __restrict__ Vt = V + (long long)t.voff * n3;
  const double gs = grad ? t.g2h3 : 0.0;
  if (t.ti == TM && t.tj == TM) {
    if (t.diag)
      accum_tile<R, TM, VEC, 2, COH>(psi, Vt, vx, oc, t.i0, TM, t.j0, TM, 1, t.c, gs, n3, r);
    else
      accum_tile<R, TM, VEC, 1, COH>(psi, Vt, vx, oc, t.i0, TM, t.j0, TM, 0, t.c, gs, n3, r);
  } else {
    accum_tile<R, TM, VEC, 0, COH>(psi, Vt, vx, oc, t.i0, t.ti, t.j0, t.tj, t.diag, t.c, gs, n3, r);
  }
}

template <typename R, int TM, int VEC>
__global__ void __launch_bounds__(256, 2)
k_accum_batch(const R* const* __restrict__ psi_tab, const R* __restrict__ V,
              double* const* __restrict__ vx_tab, const double* __restrict__ occ,
              const TileDesc* __restrict__ tiles, int grad, long long n3) {
  accum_batch_unit<R, TM, VEC, false>(psi_tab, V, vx_tab, occ, tiles, grad, n3, blockIdx.x,
                                      blockIdx.y, blockDim.x);
}

}  // namespace exx
