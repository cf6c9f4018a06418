// Persistent batched kernel: one launch per grid size runs every pass of
// every pair tile of the molecules of a batch group (exx_batch_* with
// exx_batch_set_persistent).
//
// The work of a group is a queue of items, ordered in segments: one segment
// per (wave, pass), a wave holding at most one pair tile of each molecule
// (as in the launch-per-pass schedule), the passes being
//   F  fwd_xy   (z-slab, pair)       co-density, x and y forward transforms
//   Z  zconv    (column block, kx, pair)  z transforms, kernel multiply, energy
//   E  pair energies (warps of pairs)     E_ij from the zconv partials
//   I  inv_yx   (z-slab, pair)       y and x inverse transforms: V_ij
//   A  accumulation (point block, tile)   (Vx psi) or gradient, FP64
// Waves alternate between two workspace slots.  Segments go in the order
// F(w) F(w+1) Z(w) Z(w+1) E(w) E(w+1) I(w) I(w+1) A(w) A(w+1), w = 0, 2, ..;
// each segment names the segments that must be complete before its items
// start (Z(w): F(w) and E(w-2), whose slot it reuses; I(w): Z(w) and A(w-2);
// A(w): I(w) and A(w-1), so each molecule's accumulation keeps the tile order
// of its own plan; F(w): I(w-2), or Z(w-2) for energy-only calls).  Every
// prerequisite lies earlier in the queue, and a CTA takes items in queue
// order, so the earliest unfinished item never waits: the schedule cannot
// deadlock, whatever the number of resident CTAs.
//
// A CTA takes the next item with an atomic counter, waits (thread 0, bounded,
// acquire loads, then a CTA barrier) for its segment's prerequisites, runs the
// item with the same per-CTA code as the separate kernels, and counts it done
// (a CTA barrier, then a release reduction by thread 0).  Data written by
// other CTAs of the launch are read through L2 (ldx<true>): never from a stale
// L1 or read-only cache line.  A wait that runs out (kQueuePolls polls) sets err[0] and an
// abort flag; every later item is then skipped, so the launch ends promptly and
// the host reports EXX_ERR_TIMEOUT.
#pragma once

#include "exx_kernels.cuh"

namespace exx {

enum PassKind { P_FWD = 0, P_ZCONV = 1, P_ENERGY = 2, P_INV = 3, P_ACCUM = 4 };

// One segment of the queue: items [start, start + nitems) of one pass of one
// wave, item k running units [k per, (k+1) per) of the nunits, with the wave's
// pair and tile ranges and workspace slot.
struct QSeg {
  int start, nitems, nunits, per;
  int pass, slot;
  int pair_off, npair, tile_off, ntile;
  int dep[3];  // segments that must be complete first (-1: none)
};

struct PersistArgs {
  const float* const* psi_tab;  // orbital arrays per molecule slot
  const int4* pairs;            // (i, j, pair-energy index, molecule slot)
  const TileDesc* tiles;
  const QSeg* segs;
  int nseg, total;              // segments, items
  float2* X[2];                 // per slot: spectra
  float* V[2];                  // per slot: potentials
  double* epart[2];             // per slot: zconv energy partials
  const float* Gs;              // kernel table of the group
  const float2* tw;             // twiddles of the group
  double* Epair;
  double* const* vx_tab;        // FP64 accumulators per molecule slot
  const double* occ;
  int* qc;                      // [0] queue head, [1..nseg] done counts, [nseg+1] abort
  int* err;                     // [0] set when a wait ran out
  double h3;
  long long n3;
  int nblk;                     // accumulation point blocks per tile
  int grad, energy_only, vec2;
};

constexpr int kQueuePolls = 1 << 20;  // bound of every queue wait (x ~0.25-1 us per poll)

__device__ __forceinline__ int ld_acquire_gpu(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void red_release_gpu(int* p, int v) {
  asm volatile("red.release.gpu.global.add.s32 [%0], %1;\n" ::"l"(p), "r"(v) : "memory");
}

template <int N, int NT, int MINB, bool FOLDY>
__global__ void __launch_bounds__(NT, MINB) k_persist(const PersistArgs a) {
  constexpr int L = 2 * N, W = L < 32 ? L : 32, NYB = (L + W - 1) / W;
  constexpr int NWP = NT / 32;
  __shared__ int s_item, s_seg, s_go;
  const int tid = threadIdx.x;
  int* head = a.qc;
  int* done = a.qc + 1;
  int* abortf = a.qc + 1 + a.nseg;
  // thread 0: the CTA's current segment (its items come in increasing order,
  // so the segment only moves forward) and the last segment whose
  // prerequisites were found complete
  int cur = 0, ready = -1;
  for (;;) {
    if (tid == 0) {
      const int it = atomicAdd(head, 1);
      s_item = it;
      if (it < a.total) {
        while (cur + 1 < a.nseg && a.segs[cur + 1].start <= it) ++cur;
        const int lo = cur;
        s_seg = lo;
        int go = ld_acquire_gpu(abortf) == 0;
        if (lo == ready) {
          s_go = go;
        }
        for (int k = 0; k < 3 && go && lo != ready; ++k) {
          const int d = a.segs[lo].dep[k];
          if (d < 0) continue;
          const int need = a.segs[d].nitems;
          int polls = 0;
          while (ld_acquire_gpu(done + d) < need) {
            if (ld_acquire_gpu(abortf) != 0) {
              go = 0;
              break;
            }
            if (++polls > kQueuePolls) {
              atomicExch(a.err, 1);
              atomicExch(abortf, 1);
              go = 0;
              break;
            }
            __nanosleep(256);
          }
        }
        if (go) ready = lo;
        s_go = go;
      }
    }
    __syncthreads();  // with thread 0's acquire: the prerequisites' results are visible
    const int it = s_item;
    if (it >= a.total) break;
    const QSeg sg = a.segs[s_seg];
    const int u0 = (it - sg.start) * sg.per, u1 = min(u0 + sg.per, sg.nunits);
    for (int u = u0; u < u1 && s_go; ++u) {
      if (u > u0) __syncthreads();  // the previous unit's shared memory is free
      if (sg.pass == P_FWD) {
        const int p = u / N, z = u - p * N;
        fwd_xy_unit<float, N, NT, 0, 1, false>(nullptr, a.psi_tab, a.pairs + sg.pair_off,
                                                a.X[sg.slot], a.tw, a.n3, z, p);
      } else if (sg.pass == P_ZCONV) {
        const int yb = u % NYB, r = u / NYB, kx = r % (N + 1), p = r / (N + 1);
        if (a.energy_only)
          zconv_unit<float, N, NWP, MINB, false, FOLDY, false, true, N, false, true>(
              a.X[sg.slot], a.Gs, a.tw, a.epart[sg.slot], nullptr, a.err, yb, kx, p);
        else
          zconv_unit<float, N, NWP, MINB, false, FOLDY, false, false, N, false, true>(
              a.X[sg.slot], a.Gs, a.tw, a.epart[sg.slot], nullptr, a.err, yb, kx, p);
      } else if (sg.pass == P_ENERGY) {
        // one warp per pair: E_ij = h^3 sum of the pair's column-block partials
        const int q = u * NWP + (tid >> 5), lane = tid & 31;
        if (q < sg.npair) {
          constexpr int nper = (N + 1) * NYB;
          const double* ep = a.epart[sg.slot] + (long long)q * nper;
          double s = 0.0;
          for (int t = lane; t < nper; t += 32) s += ldx<true>(ep + t);
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
          if (lane == 0) a.Epair[a.pairs[sg.pair_off + q].z] = a.h3 * s;
        }
      } else if (sg.pass == P_INV) {
        const int p = u / N, z = u - p * N;
        inv_yx_unit<float, N, NT, 0, 1, false, true>(a.X[sg.slot], a.V[sg.slot], a.tw, z, p);
      } else {
        const int t = u / a.nblk, b = u - t * a.nblk;
        if (a.vec2)
          accum_batch_unit<float, 8, 2, true>(a.psi_tab, a.V[sg.slot], a.vx_tab, a.occ,
                                              a.tiles + sg.tile_off, a.grad, a.n3, b, t, NT);
        else
          accum_batch_unit<float, 8, 1, true>(a.psi_tab, a.V[sg.slot], a.vx_tab, a.occ,
                                              a.tiles + sg.tile_off, a.grad, a.n3, b, t, NT);
      }
    }
    __syncthreads();  // then one release by thread 0 publishes the whole CTA's results
    if (tid == 0) red_release_gpu(done + s_seg, 1);
  }
}

}  // namespace exx
