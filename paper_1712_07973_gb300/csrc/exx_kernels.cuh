// CUDA kernels of the exact-exchange pair pipeline (sm_103a).
//
// For every orbital pair (i, j) of a pair tile (arXiv 1712.07973, Sec. 2.1:
// kernel 1 co-density, kernel 2 Poisson solve, kernel 3 products):
//
//   fwd_xy  (one CTA per z-slab and pair)
//           rho = psi_i psi_j on the slab, real-to-complex FFT of length 2n
//           along x with x >= n zero (two real lines packed per complex
//           line), then the pruned complex FFT of length 2n along y with
//           y >= n zero.  Writes X2[pair][kx][z][ky], kx in [0, n].
//   zconv   (one CTA per 32 columns (kx, ky) and pair)
//           along z: pruned forward FFT (z >= n zero), multiply by the real
//           kernel spectrum Ghat (Sec. 2.1.2; scaled by 1/(2n)^3), Parseval
//           energy sum w(kx) Ghat |rho_hat|^2, inverse FFT keeping z < n.
//           In place on X2 (becomes X3).
//   inv_yx  (one CTA per z-slab and pair)
//           inverse FFT along y keeping y < n, complex-to-real FFT along x
//           keeping x < n: V_ij on the n^3 mesh.
//   accum   (grid-stride over mesh points, one pair tile)
//           (Vx psi)_i += -alpha f_j V_ij psi_j and, for i != j,
//           (Vx psi)_j += -alpha f_i V_ij psi_i (Eq. daction); FP32 sums
//           over the tile, FP64 accumulation across tiles, deterministic.
//
// Layouts: psi[o][z][y][x]; X2/X3[p][kx][z][ky] complex; V[p][z][y][x].
#pragma once

#include "exx_fft.cuh"

namespace exx {

// Padded scratch layout of one line in the [a][k1] form of the four-step:
// slot(a, k1) = a * (L1 + 1) + k1; the line stride is odd so that lines of
// different units land on different banks.
template <int L1, int L2> struct Scr {
  static constexpr int row = L1 + 1;
  static constexpr int line = (L2 * row) | 1;
};

template <typename R> __device__ __forceinline__ R sq(R a) { return a * a; }

// ------------------------------------------------------------------ fwd_xy
template <typename R, int N, int NT, int Q>
__global__ void __launch_bounds__(NT)
k_fwd_xy(const R* __restrict__ psi, const int4* __restrict__ pairs, cplx<R>* __restrict__ X2,
         const cplx<R>* __restrict__ tw_g, long long n3) {
  using C = cplx<R>;
  constexpr int L = 2 * N, L1 = split_l1(L), L2 = L / L1, H1 = L1 / 2;
  constexpr int NH = (N + 1) / 2;  // packed line pairs
  using S_ = Scr<L1, L2>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* tw = reinterpret_cast<C*>(smem_raw);
  C* Sl = tw + L;                       // [(N+1)][N]
  C* S = Sl + (N + 1) * N;              // [Q][line]
  R* stg = reinterpret_cast<R*>(S + Q * S_::line);  // [2Q][N]

  const int tid = threadIdx.x;
  const int z = blockIdx.x;
  const int p = blockIdx.y;
  const int4 pr = pairs[p];
  const R* __restrict__ pi = psi + (long long)pr.x * n3 + (long long)z * N * N;
  const R* __restrict__ pj = psi + (long long)pr.y * n3 + (long long)z * N * N;
  for (int t = tid; t < L; t += NT) tw[t] = tw_g[t];

  // ---- x: real-to-complex, two lines (y, y+1) packed as re + i im
  for (int q0 = 0; q0 < NH; q0 += Q) {
    const int nq = min(Q, NH - q0);
    for (int idx = tid; idx < 2 * Q * N; idx += NT) {
      const int r = idx / N, x = idx - r * N;
      const int y = 2 * q0 + r;
      stg[idx] = (r < 2 * nq && y < N) ? pi[y * N + x] * pj[y * N + x] : R(0);
    }
    __syncthreads();
    for (int u = tid; u < nq * L2; u += NT) {
      const int qq = u / L2, n2 = u - qq * L2;
      C v[L1];
#pragma unroll
      for (int n1 = 0; n1 < H1; ++n1) {
        const int x = L2 * n1 + n2;
        v[n1] = mkc<C>(stg[(2 * qq) * N + x], stg[(2 * qq + 1) * N + x]);
      }
      dft_halfin<L1, -1>(v);
      C* s = S + qq * S_::line + n2 * S_::row;
      s[0] = v[0];
#pragma unroll
      for (int k1 = 1; k1 < L1; ++k1) s[k1] = cmul(v[k1], tw[n2 * k1]);
    }
    __syncthreads();
    for (int u = tid; u < nq * L1; u += NT) {
      const int qq = u / L1, k1 = u - qq * L1;
      C v[L2];
      C* s = S + qq * S_::line + k1;
#pragma unroll
      for (int n2 = 0; n2 < L2; ++n2) v[n2] = s[n2 * S_::row];
      dft<L2, 1, -1>(v);
#pragma unroll
      for (int k2 = 0; k2 < L2; ++k2) s[k2 * S_::row] = v[k2];
    }
    __syncthreads();
    // unpack the two real lines: A = (C[k] + conj C[L-k]) / 2,
    //                            B = (C[k] - conj C[L-k]) / (2i)
    for (int u = tid; u < (N + 1) * nq; u += NT) {
      const int k = u / nq, qq = u - k * nq;
      const int km = (L - k) % L;
      const C* s = S + qq * S_::line;
      const C c = s[(k / L1) * S_::row + (k % L1)];
      const C d = s[(km / L1) * S_::row + (km % L1)];
      const C A = mkc<C>(R(0.5) * (c.x + d.x), R(0.5) * (c.y - d.y));
      const C B = mkc<C>(R(0.5) * (c.y + d.y), R(-0.5) * (c.x - d.x));
      const int y = 2 * (q0 + qq);
      Sl[k * N + y] = A;
      if (y + 1 < N) Sl[k * N + y + 1] = B;
    }
    __syncthreads();
  }

  // ---- y: pruned forward FFT per kx row, straight to global memory
  for (int r0 = 0; r0 <= N; r0 += Q) {
    const int nr = min(Q, N + 1 - r0);
    for (int u = tid; u < nr * L2; u += NT) {
      const int r = u / L2, n2 = u - r * L2;
      const C* row = Sl + (r0 + r) * N;
      C v[L1];
#pragma unroll
      for (int n1 = 0; n1 < H1; ++n1) v[n1] = row[L2 * n1 + n2];
      dft_halfin<L1, -1>(v);
      C* s = S + r * S_::line + n2 * S_::row;
      s[0] = v[0];
#pragma unroll
      for (int k1 = 1; k1 < L1; ++k1) s[k1] = cmul(v[k1], tw[n2 * k1]);
    }
    __syncthreads();
    for (int u = tid; u < nr * L1; u += NT) {
      const int r = u / L1, k1 = u - r * L1;
      C v[L2];
      const C* s = S + r * S_::line + k1;
#pragma unroll
      for (int n2 = 0; n2 < L2; ++n2) v[n2] = s[n2 * S_::row];
      dft<L2, 1, -1>(v);
      C* out = X2 + (((long long)p * (N + 1) + (r0 + r)) * N + z) * L + k1;
#pragma unroll
      for (int k2 = 0; k2 < L2; ++k2) out[L1 * k2] = v[k2];
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------- zconv
template <typename R, int N, int NW, bool ENERGY_ONLY>
__global__ void __launch_bounds__(32 * NW)
k_zconv(cplx<R>* __restrict__ X, const R* __restrict__ Gs, const cplx<R>* __restrict__ tw_g,
        double* __restrict__ epart) {
  using C = cplx<R>;
  constexpr int L = 2 * N, L1 = split_l1(L), L2 = L / L1, H1 = L1 / 2;
  constexpr int W = L < 32 ? L : 32;
  constexpr int M = N + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* tw = reinterpret_cast<C*>(smem_raw);
  C* buf = tw + L;  // [L slots][W]
  __shared__ double red[NW];

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int yb = blockIdx.x, kx = blockIdx.y, p = blockIdx.z;
  const int ky = yb * W + lane;
  const bool valid = lane < W && ky < L;
  for (int t = tid; t < L; t += 32 * NW) tw[t] = tw_g[t];
  C* col = X + (((long long)p * M + kx) * N) * L + (valid ? ky : 0);
  __syncthreads();

  // forward, pass 1: L2 pruned DFTs of length L1 over z = L2 n1 + n2
  for (int n2 = warp; n2 < L2; n2 += NW) {
    C v[L1];
#pragma unroll
    for (int n1 = 0; n1 < H1; ++n1)
      v[n1] = valid ? col[(long long)(L2 * n1 + n2) * L] : mkc<C>(R(0), R(0));
    dft_halfin<L1, -1>(v);
    if (lane < W) {
      buf[(n2 * L1) * W + lane] = v[0];
#pragma unroll
      for (int k1 = 1; k1 < L1; ++k1) buf[(n2 * L1 + k1) * W + lane] = cmul(v[k1], tw[n2 * k1]);
    }
  }
  __syncthreads();

  // pass 2 of the forward, kernel multiply, pass 1 of the inverse
  const int kyf = ky <= N ? ky : L - ky;
  const R* __restrict__ Gk = Gs + (long long)kx * M * M + (valid ? kyf : 0);
  double eacc = 0.0;
  for (int k1 = warp; k1 < L1; k1 += NW) {
    C v[L2];
#pragma unroll
    for (int n2 = 0; n2 < L2; ++n2) v[n2] = lane < W ? buf[(n2 * L1 + k1) * W + lane] : mkc<C>(R(0), R(0));
    dft<L2, 1, -1>(v);
    R es = R(0);
#pragma unroll
    for (int k2 = 0; k2 < L2; ++k2) {
      const int kz = k1 + L1 * k2;
      const int kzf = kz <= N ? kz : L - kz;
      const R g = valid ? __ldg(Gk + kzf * M) : R(0);
      es += g * (sq(v[k2].x) + sq(v[k2].y));
      v[k2] = cscale(v[k2], g);
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
    // inverse, pass 2: L2 DFTs of length L1, only z = L2 m1 + m2 < n kept
    for (int m2 = warp; m2 < L2; m2 += NW) {
      C v[L1];
#pragma unroll
      for (int k1 = 0; k1 < L1; ++k1) v[k1] = lane < W ? buf[(m2 * L1 + k1) * W + lane] : mkc<C>(R(0), R(0));
      dft_halfout<L1, 1>(v);
      if (valid) {
#pragma unroll
        for (int m1 = 0; m1 < H1; ++m1) col[(long long)(L2 * m1 + m2) * L] = v[m1];
      }
    }
  }
  // Parseval energy of this block (fixed-order reduction)
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) eacc += __shfl_xor_sync(0xffffffffu, eacc, o);
  if (lane == 0) red[warp] = eacc;
  __syncthreads();
  if (tid == 0) {
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < NW; ++w) s += red[w];
    const double wk = (kx == 0 || kx == N) ? 1.0 : 2.0;
    epart[((long long)p * M + kx) * gridDim.x + yb] = wk * s;
  }
}

// ------------------------------------------------------------------ inv_yx
template <typename R, int N, int NT, int Q>
__global__ void __launch_bounds__(NT)
k_inv_yx(const cplx<R>* __restrict__ X3, R* __restrict__ V, const cplx<R>* __restrict__ tw_g) {
  using C = cplx<R>;
  constexpr int L = 2 * N, L1 = split_l1(L), L2 = L / L1, H1 = L1 / 2;
  constexpr int NH = (N + 1) / 2;
  using S_ = Scr<L1, L2>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* tw = reinterpret_cast<C*>(smem_raw);
  C* Sl = tw + L;           // [(N+1)][N]
  C* S = Sl + (N + 1) * N;  // [Q][line]

  const int tid = threadIdx.x;
  const int z = blockIdx.x;
  const int p = blockIdx.y;
  for (int t = tid; t < L; t += NT) tw[t] = tw_g[t];
  __syncthreads();

  // ---- y: inverse FFT per kx row, keep y < n
  for (int r0 = 0; r0 <= N; r0 += Q) {
    const int nr = min(Q, N + 1 - r0);
    for (int u = tid; u < nr * L1; u += NT) {
      const int r = u / L1, k1 = u - r * L1;
      const C* in = X3 + (((long long)p * (N + 1) + (r0 + r)) * N + z) * L + k1;
      C v[L2];
#pragma unroll
      for (int k2 = 0; k2 < L2; ++k2) v[k2] = in[L1 * k2];
      dft<L2, 1, 1>(v);
      C* s = S + r * S_::line + k1;
      s[0] = v[0];
#pragma unroll
      for (int m2 = 1; m2 < L2; ++m2) s[m2 * S_::row] = cmulc(v[m2], tw[m2 * k1]);
    }
    __syncthreads();
    for (int u = tid; u < nr * L2; u += NT) {
      const int r = u / L2, m2 = u - r * L2;
      const C* s = S + r * S_::line + m2 * S_::row;
      C v[L1];
#pragma unroll
      for (int k1 = 0; k1 < L1; ++k1) v[k1] = s[k1];
      dft_halfout<L1, 1>(v);
      C* row = Sl + (r0 + r) * N;
#pragma unroll
      for (int m1 = 0; m1 < H1; ++m1) row[L2 * m1 + m2] = v[m1];
    }
    __syncthreads();
  }

  // ---- x: complex-to-real, two lines packed: C[k] = A[k] + i B[k] with the
  //      Hermitian extension A[L-k] = conj A[k]; real parts of A, B are the lines
  for (int q0 = 0; q0 < NH; q0 += Q) {
    const int nq = min(Q, NH - q0);
    for (int u = tid; u < nq * L1; u += NT) {
      const int k1 = u / nq, qq = u - k1 * nq;
      const int y = 2 * (q0 + qq);
      C v[L2];
#pragma unroll
      for (int k2 = 0; k2 < L2; ++k2) {
        const int k = k1 + L1 * k2;
        const int kk = k <= N ? k : L - k;
        C a = Sl[kk * N + y];
        C b = (y + 1 < N) ? Sl[kk * N + y + 1] : mkc<C>(R(0), R(0));
        if (kk == 0 || kk == N) {
          a.y = R(0);
          b.y = R(0);
        }
        if (k > N) {
          a.y = -a.y;
          b.y = -b.y;
        }
        v[k2] = mkc<C>(a.x - b.y, a.y + b.x);
      }
      dft<L2, 1, 1>(v);
      C* s = S + qq * S_::line + k1;
      s[0] = v[0];
#pragma unroll
      for (int m2 = 1; m2 < L2; ++m2) s[m2 * S_::row] = cmulc(v[m2], tw[m2 * k1]);
    }
    __syncthreads();
    for (int u = tid; u < nq * L2; u += NT) {
      const int qq = u / L2, m2 = u - qq * L2;
      const C* s = S + qq * S_::line + m2 * S_::row;
      C v[L1];
#pragma unroll
      for (int k1 = 0; k1 < L1; ++k1) v[k1] = s[k1];
      dft_halfout<L1, 1>(v);
      const int y = 2 * (q0 + qq);
      R* out = V + ((long long)p * N + z) * N * N + (long long)y * N;
#pragma unroll
      for (int m1 = 0; m1 < H1; ++m1) {
        const int x = L2 * m1 + m2;
        out[x] = v[m1].x;
        if (y + 1 < N) out[N + x] = v[m1].y;
      }
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------- accum
// One pair tile: orbitals i0..i0+ti-1 (block I) and j0..j0+tj-1 (block J);
// off-diagonal tiles hold all ti*tj pairs (slot a*tj + b), diagonal tiles
// (I == J) the ti(ti+1)/2 pairs a <= b in row-major order.
template <typename R, int TM>
__global__ void __launch_bounds__(256)
k_accum(const R* __restrict__ psi, const R* __restrict__ V, double* __restrict__ vx,
        const double* __restrict__ occ, int i0, int ti, int j0, int tj, int diag, double c,
        long long n3) {
  R fi[TM], fj[TM];
#pragma unroll
  for (int a = 0; a < TM; ++a) {
    fi[a] = a < ti ? (R)occ[i0 + a] : R(0);
    fj[a] = a < tj ? (R)occ[j0 + a] : R(0);
  }
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n3;
       r += (long long)gridDim.x * blockDim.x) {
    R pi[TM], pj[TM], ai[TM], aj[TM];
#pragma unroll
    for (int a = 0; a < TM; ++a) {
      pi[a] = a < ti ? psi[(long long)(i0 + a) * n3 + r] : R(0);
      pj[a] = (!diag && a < tj) ? psi[(long long)(j0 + a) * n3 + r] : pi[a];
      ai[a] = R(0);
      aj[a] = R(0);
    }
#pragma unroll
    for (int a = 0; a < TM; ++a) {
      if (a >= ti) continue;
#pragma unroll
      for (int b = 0; b < TM; ++b) {
        if (b >= tj) continue;
        if (diag && b < a) continue;
        const int slot = diag ? a * tj - (a * (a - 1)) / 2 + (b - a) : a * tj + b;
        const R v = V[(long long)slot * n3 + r];
        ai[a] += fj[b] * v * pj[b];
        if (!(diag && a == b)) aj[b] += fi[a] * v * pi[a];
      }
    }
    if (diag) {
#pragma unroll
      for (int a = 0; a < TM; ++a)
        if (a < ti) vx[(long long)(i0 + a) * n3 + r] += c * ((double)ai[a] + (double)aj[a]);
    } else {
#pragma unroll
      for (int a = 0; a < TM; ++a)
        if (a < ti) vx[(long long)(i0 + a) * n3 + r] += c * (double)ai[a];
#pragma unroll
      for (int b = 0; b < TM; ++b)
        if (b < tj) vx[(long long)(j0 + b) * n3 + r] += c * (double)aj[b];
    }
  }
}

}  // namespace exx
