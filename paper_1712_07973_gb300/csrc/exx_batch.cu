// Batched exact exchange over many molecules of uneven size (declared in
// include/exx.h): exx_batch_create / exx_batch_set_buffers / exx_batch_apply /
// exx_batch_energy / exx_batch_graph / exx_batch_info / exx_batch_destroy.
//
// Molecules with the same (n, h, kernel) form a group that shares the kernel
// spectrum, the twiddles and the compiled kernels.  Within a group the pair
// tiles of all molecules are scheduled in waves: a wave takes at most one
// tile of each molecule (round-robin, under a budget of pair solves), so every
// launch of the pipeline processes pairs of many molecules at once while the
// tiles of one wave never touch the same accumulator; each molecule's tiles run
// in their own order, so the FP64 accumulation is deterministic and equal to
// the single-molecule plan's.  The whole enqueue sequence of a call can be
// captured once into a CUDA graph and replayed.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <string>
#include <vector>

#include "exx.h"
#include "exx_ops.cuh"

namespace exx_host {
bool kernel_spectrum_octant(int n, double h, int kind, double omega, double* out);
}

namespace exx {
const Ops* find_ops(int prec, int n);
__global__ void k_pair_energy(const double* __restrict__ epart, int nper,
                              const int4* __restrict__ pairs, int npair, double h3,
                              double* __restrict__ Epair);

struct MolTot {
  int N;
  int occ_off;
  long long ep_off;  // first pair energy of the molecule in Epair
  double alpha;
};

// E_x of every molecule (one block per molecule, fixed-order reduction)
__global__ void k_exx_total_batch(const double* __restrict__ Epair, const MolTot* __restrict__ mt,
                                  const double* __restrict__ occ, double* __restrict__ E) {
  __shared__ double red[256];
  const MolTot m = mt[blockIdx.x];
  const double* oc = occ + m.occ_off;
  const double* ep = Epair + m.ep_off;
  double s = 0.0;
  // pair g -> (i, j): walk rows (N is small here: up to a few hundred)
  for (int i = 0; i < m.N; ++i) {
    const long long row = (long long)i * m.N - ((long long)i * (i - 1)) / 2;
    for (int j = i + threadIdx.x; j < m.N; j += blockDim.x) {
      const double w = (i == j) ? 1.0 : 2.0;
      s += w * oc[i] * oc[j] * ep[row + (j - i)];
    }
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) E[blockIdx.x] = -0.5 * m.alpha * red[0];
}

// FP64 accumulators to the callers' float outputs (grid.y = molecule)
__global__ void k_to_float_batch(double* const* __restrict__ src, float* const* __restrict__ dst,
                                 const long long* __restrict__ count) {
  const double* a = src[blockIdx.y];
  float* b = dst[blockIdx.y];
  const long long n = count[blockIdx.y];
  if (b == nullptr) return;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}
}  // namespace exx

using namespace exx;

namespace {

struct Wave {
  int pair_off, npair;
  int tile_off, ntile;
};

struct Group {
  int n = 0, kind = 0;
  double h = 0.0;
  const Ops* ops = nullptr;
  std::vector<int> mols;
  std::vector<Wave> waves;
  void* Gs = nullptr;
  void* tw = nullptr;
  CUtensorMap gmap{};  // TMA descriptor of Gs (ops->stage_table)
  // persistent mode: the group's queue segments (offset into the batch's
  // segment table and count, per mode: 0 apply or gradient, 1 energy), items,
  // and accumulation point blocks per tile
  int seg_off[2] = {0, 0}, nseg[2] = {0, 0}, total[2] = {0, 0};
  int nblk = 0;
};

struct Mol {
  int n, N, T, group;
  double h, alpha;
  int occ_off;
  long long ep_off, P;
  long long vacc_off;  // into the FP64 accumulator block
};

const long long kWavePairBudget = 512;  // pair solves per wave (bounds the workspace)

}  // namespace

struct exx_batch_s {
  int nmol = 0, kind = 0;
  std::vector<Mol> mol;
  std::vector<Group> groups;
  std::vector<int4> pairs;
  std::vector<TileDesc> tiles;
  size_t ws = 0;
  int max_wave_pairs = 0;
  size_t x_bytes = 0, v_bytes = 0, ep_bytes = 0;
  // device
  int4* d_pairs = nullptr;
  TileDesc* d_tiles = nullptr;
  double* d_occ = nullptr;
  double* Epair = nullptr;
  double* epart = nullptr;
  int* d_err = nullptr;  // set by a device-side wait that ran out
  void* X = nullptr;
  void* V = nullptr;
  double* vacc = nullptr;
  MolTot* d_mt = nullptr;
  const float** d_psi_tab = nullptr;
  double** d_vacc_tab = nullptr;
  float** d_vx_tab = nullptr;
  long long* d_count = nullptr;
  bool have_vx = false;
  bool buffers_set = false;
  bool vec2 = true;  // every orbital array 8-byte aligned: paired loads in accum
  // second pipeline lane (as in a single plan): its workspaces, streams, events
  int lanes = 1;
  double* epart2 = nullptr;
  void* X_2 = nullptr;
  void* V_2 = nullptr;
  cudaStream_t ls[2] = {nullptr, nullptr};
  cudaEvent_t ev_fork = nullptr, ev_done[2] = {nullptr, nullptr}, ev_free[2] = {nullptr, nullptr};
  // graph capture
  bool graph_on = false;
  // persistent mode (exx_batch_set_persistent): queue segments of every group,
  // their device copy and the queue counters
  bool persistent = false;
  std::vector<QSeg> segs;
  QSeg* d_segs = nullptr;
  int* d_qc = nullptr;
  int qc_len = 0;
  cudaGraphExec_t gexec[3] = {nullptr, nullptr, nullptr};  // [apply, energy, gradient]
  double* gE[3] = {nullptr, nullptr, nullptr};
  cudaStream_t gstream[3] = {nullptr, nullptr, nullptr};
  std::string err;
};

namespace {

void batch_free(exx_batch_t b) {
  void* ptrs[] = {b->d_pairs, b->d_tiles, b->d_occ,  b->Epair,           b->epart,
                  b->X,       b->V,       b->vacc,   b->d_mt,            (void*)b->d_psi_tab,
                  b->d_vacc_tab, b->d_vx_tab, b->d_count, b->d_err, b->d_segs, b->d_qc};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  for (Group& g : b->groups) {
    if (g.Gs) cudaFree(g.Gs);
    if (g.tw) cudaFree(g.tw);
  }
  for (int k = 0; k < 3; ++k)
    if (b->gexec[k]) cudaGraphExecDestroy(b->gexec[k]);
  for (void* q : {static_cast<void*>(b->epart2), b->X_2, b->V_2})
    if (q) cudaFree(q);
  for (int l = 0; l < 2; ++l) {
    if (b->ls[l]) cudaStreamDestroy(b->ls[l]);
    if (b->ev_done[l]) cudaEventDestroy(b->ev_done[l]);
    if (b->ev_free[l]) cudaEventDestroy(b->ev_free[l]);
  }
  if (b->ev_fork) cudaEventDestroy(b->ev_fork);
}

template <typename T> bool balloc(exx_batch_t b, T** p, size_t bytes) {
  void* q = nullptr;
  if (cudaMalloc(&q, bytes ? bytes : 16) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  b->ws += bytes;
  *p = static_cast<T*>(q);
  return true;
}

// apply: Vx psi (grad = false) or the gradient 2 f_k h^3 (Vx psi)_k (grad =
// true) into the bound outputs
// Queue segments of a group for the persistent kernel (order and
// prerequisites in exx_persist.cuh); indices are relative to the group's
// first segment.  stall: test hook, one extra segment that never completes is
// made a prerequisite of the first zconv segment.
void build_segments(exx_batch_t b, Group& g, bool apply, bool stall, std::vector<QSeg>& out) {
  const int n = g.n, W = (int)g.waves.size();
  const int NWP = g.ops->persist_nt / 32;
  const long long n3 = (long long)n * n * n;
  g.nblk = (int)((n3 + g.ops->persist_nt - 1) / g.ops->persist_nt);
  std::vector<int> idx((size_t)W * 5, -1);
  std::vector<QSeg> v;
  int cursor = 0;
  const int passes_apply[5] = {P_FWD, P_ZCONV, P_ENERGY, P_INV, P_ACCUM};
  const int np = apply ? 5 : 3;
  for (int w0 = 0; w0 < W; w0 += 2)
    for (int k = 0; k < np; ++k)
      for (int w = w0; w < std::min(W, w0 + 2); ++w) {
        const int ps = passes_apply[k];
        const Wave& wv = g.waves[w];
        QSeg q;
        q.start = cursor;
        q.pass = ps;
        q.slot = w % 2;
        q.pair_off = wv.pair_off;
        q.npair = wv.npair;
        q.tile_off = wv.tile_off;
        q.ntile = wv.ntile;
        q.nunits = ps == P_FWD || ps == P_INV ? wv.npair * n
                   : ps == P_ZCONV            ? wv.npair * (n + 1) * g.ops->nyb
                   : ps == P_ENERGY           ? (wv.npair + NWP - 1) / NWP
                                              : wv.ntile * g.nblk;
        // units per item: small grids take several, so that the per-item queue
        // work (counter, barriers, release) stays small against the transforms
        q.per = (ps == P_FWD || ps == P_INV || ps == P_ZCONV) ? (n <= 48 ? 4 : n <= 80 ? 2 : 1) : 1;
        q.nitems = (q.nunits + q.per - 1) / q.per;
        q.dep[0] = q.dep[1] = q.dep[2] = -1;
        auto at = [&](int ww, int pp) { return ww >= 0 ? idx[(size_t)ww * 5 + pp] : -1; };
        if (ps == P_FWD) {
          q.dep[0] = at(w - 2, apply ? P_INV : P_ZCONV);  // its workspace slot is free
        } else if (ps == P_ZCONV) {
          q.dep[0] = at(w, P_FWD);
          q.dep[1] = at(w - 2, P_ENERGY);  // energy partials of the slot read
        } else if (ps == P_ENERGY) {
          q.dep[0] = at(w, P_ZCONV);
        } else if (ps == P_INV) {
          q.dep[0] = at(w, P_ZCONV);
          q.dep[1] = at(w - 2, P_ACCUM);  // potentials of the slot read
        } else {
          q.dep[0] = at(w, P_INV);
          q.dep[1] = at(w - 1, P_ACCUM);  // accumulation in tile order
        }
        idx[(size_t)w * 5 + ps] = (int)v.size();
        v.push_back(q);
        cursor += q.nitems;
      }
  const int m = apply ? 0 : 1;
  g.total[m] = cursor;
  if (stall) {  // never completes: no item maps to it
    QSeg q{};
    q.start = cursor;
    q.nunits = q.nitems = q.per = 1;
    q.pass = P_FWD;
    q.dep[0] = q.dep[1] = q.dep[2] = -1;
    v[idx[P_ZCONV]].dep[2] = (int)v.size();
    v.push_back(q);
  }
  g.seg_off[m] = (int)out.size();
  g.nseg[m] = (int)v.size();
  out.insert(out.end(), v.begin(), v.end());
  (void)b;
}

exx_status_t enqueue(exx_batch_t b, double* E_dev, bool apply, bool grad, cudaStream_t st) {
  if (apply) {
    long long tot = 0;
    for (const Mol& m : b->mol) tot += (long long)m.N * m.n * m.n * m.n;
    if (cudaMemsetAsync(b->vacc, 0, (size_t)tot * sizeof(double), st) != cudaSuccess) return EXX_ERR_CUDA;
  }
  // two lanes: consecutive waves alternate between two streams with their own
  // workspaces; the accumulation stays on st in wave order
  // persistent mode: one launch per group that supports it, all on st (the
  // queue uses both workspace slots, so no lanes)
  const int nl = b->persistent ? 1 : b->lanes;
  if (nl > 1) {
    if (cudaEventRecord(b->ev_fork, st) != cudaSuccess) return EXX_ERR_CUDA;
    for (int l = 0; l < nl; ++l)
      if (cudaStreamWaitEvent(b->ls[l], b->ev_fork, 0) != cudaSuccess) return EXX_ERR_CUDA;
  }
  void* Xl[2] = {b->X, b->X_2};
  void* Vl[2] = {b->V, b->V_2};
  double* epl[2] = {b->epart, b->epart2};
  bool used[2] = {false, false};
  int k = 0;
  for (const Group& g : b->groups) {
    const long long n3 = (long long)g.n * g.n * g.n;
    if (b->persistent && g.ops->persist_ok) {
      const int m = apply ? 0 : 1;
      if (cudaMemsetAsync(b->d_qc, 0, (size_t)(g.nseg[m] + 2) * sizeof(int), st) != cudaSuccess)
        return EXX_ERR_CUDA;
      PersistArgs a{};
      a.psi_tab = b->d_psi_tab;
      a.pairs = b->d_pairs;
      a.tiles = b->d_tiles;
      a.segs = b->d_segs + g.seg_off[m];
      a.nseg = g.nseg[m];
      a.total = g.total[m];
      a.X[0] = static_cast<float2*>(b->X);
      a.X[1] = static_cast<float2*>(b->X_2);
      a.V[0] = static_cast<float*>(b->V);
      a.V[1] = static_cast<float*>(b->V_2);
      a.epart[0] = b->epart;
      a.epart[1] = b->epart2;
      a.Gs = static_cast<const float*>(g.Gs);
      a.tw = static_cast<const float2*>(g.tw);
      a.Epair = b->Epair;
      a.vx_tab = b->d_vacc_tab;
      a.occ = b->d_occ;
      a.qc = b->d_qc;
      a.err = b->d_err;
      a.h3 = g.h * g.h * g.h;
      a.n3 = n3;
      a.nblk = g.nblk;
      a.grad = grad ? 1 : 0;
      a.energy_only = apply ? 0 : 1;
      a.vec2 = (b->vec2 && (n3 % 2) == 0) ? 1 : 0;
      if (g.ops->persist(a, st) != cudaSuccess) return EXX_ERR_CUDA;
      continue;
    }
    const int nper = (g.n + 1) * g.ops->nyb;
    const double h3 = g.h * g.h * g.h;
    for (const Wave& w : g.waves) {
      const int4* pr = b->d_pairs + w.pair_off;
      const int l = nl > 1 ? (k++ & 1) : 0;
      cudaStream_t sl = nl > 1 ? b->ls[l] : st;
      g.ops->fwd_xy(nullptr, reinterpret_cast<const void* const*>(b->d_psi_tab), pr, w.npair, Xl[l],
                    g.tw, n3, sl);
      g.ops->zconv(Xl[l], g.Gs, g.tw, &g.gmap, epl[l], b->d_err, w.npair, !apply, sl);
      k_pair_energy<<<(w.npair * 32 + 255) / 256, 256, 0, sl>>>(epl[l], nper, pr, w.npair, h3,
                                                                 b->Epair);
      if (apply) {
        if (nl > 1 && used[l] && cudaStreamWaitEvent(sl, b->ev_free[l], 0) != cudaSuccess)
          return EXX_ERR_CUDA;
        g.ops->inv_yx(Xl[l], Vl[l], g.tw, w.npair, sl);
        if (nl > 1 && (cudaEventRecord(b->ev_done[l], sl) != cudaSuccess ||
                       cudaStreamWaitEvent(st, b->ev_done[l], 0) != cudaSuccess))
          return EXX_ERR_CUDA;
        used[l] = true;
        const bool v2 = b->vec2 && (n3 % 2) == 0;
        const int threads = 256;
        const long long blocks = (n3 / (v2 ? 2 : 1) + threads - 1) / threads;
        if (v2)
          k_accum_batch<float, 8, 2><<<dim3((unsigned)blocks, w.ntile), threads, 0, st>>>(
              b->d_psi_tab, static_cast<const float*>(Vl[l]), b->d_vacc_tab, b->d_occ,
              b->d_tiles + w.tile_off, grad ? 1 : 0, n3);
        else
          k_accum_batch<float, 8, 1><<<dim3((unsigned)blocks, w.ntile), threads, 0, st>>>(
              b->d_psi_tab, static_cast<const float*>(Vl[l]), b->d_vacc_tab, b->d_occ,
              b->d_tiles + w.tile_off, grad ? 1 : 0, n3);
        if (nl > 1 && cudaEventRecord(b->ev_free[l], st) != cudaSuccess) return EXX_ERR_CUDA;
      }
    }
  }
  if (nl > 1)  // join both lanes
    for (int l = 0; l < nl; ++l)
      if (cudaEventRecord(b->ev_done[l], b->ls[l]) != cudaSuccess ||
          cudaStreamWaitEvent(st, b->ev_done[l], 0) != cudaSuccess)
        return EXX_ERR_CUDA;
  k_exx_total_batch<<<b->nmol, 256, 0, st>>>(b->Epair, b->d_mt, b->d_occ, E_dev);
  if (apply && b->have_vx) {
    long long mx = 0;
    for (const Mol& m : b->mol) mx = std::max(mx, (long long)m.N * m.n * m.n * m.n);
    const long long blocks = std::min<long long>((mx + 255) / 256, 1024);
    k_to_float_batch<<<dim3((unsigned)blocks, b->nmol), 256, 0, st>>>(b->d_vacc_tab, b->d_vx_tab,
                                                                       b->d_count);
  }
  return cudaGetLastError() == cudaSuccess ? EXX_OK : EXX_ERR_CUDA;
}

exx_status_t run_batch(exx_batch_t b, double* E_dev, bool apply, bool grad, cudaStream_t st) {
  if (!b->buffers_set) return EXX_ERR_INVALID_ARG;
  if (apply && !b->have_vx) return EXX_ERR_INVALID_ARG;
  const int k = apply ? (grad ? 2 : 0) : 1;
  if (!b->graph_on) return enqueue(b, E_dev, apply, grad, st);
  if (st == nullptr) return EXX_ERR_INVALID_ARG;  // capture needs a created stream
  if (b->gexec[k] && (b->gE[k] != E_dev || b->gstream[k] != st)) {
    cudaGraphExecDestroy(b->gexec[k]);
    b->gexec[k] = nullptr;
  }
  if (!b->gexec[k]) {
    if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      cudaGetLastError();
      return EXX_ERR_CUDA;
    }
    exx_status_t s = enqueue(b, E_dev, apply, grad, st);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(st, &graph);
    if (s != EXX_OK || e != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      return EXX_ERR_CUDA;
    }
    e = cudaGraphInstantiate(&b->gexec[k], graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      cudaGetLastError();
      b->gexec[k] = nullptr;
      return EXX_ERR_CUDA;
    }
    b->gE[k] = E_dev;
    b->gstream[k] = st;
  }
  return cudaGraphLaunch(b->gexec[k], st) == cudaSuccess ? EXX_OK : EXX_ERR_CUDA;
}

int default_tile(int N, int requested) {
  int T = requested > 0 ? requested : 8;
  if (T > 8) T = 8;
  return T < N ? T : N;
}

}  // namespace

extern "C" {

exx_status_t exx_batch_create(exx_batch_t* out, int nmol, const exx_mol_desc* mols, int kernel,
                              void* cuda_stream) {
  if (out == nullptr) return EXX_ERR_INVALID_ARG;
  *out = nullptr;
  if (nmol < 1 || mols == nullptr) return EXX_ERR_INVALID_ARG;
  if (kernel != EXX_KERNEL_SINC && kernel != EXX_KERNEL_HOCKNEY) return EXX_ERR_INVALID_ARG;
  for (int m = 0; m < nmol; ++m) {
    const exx_mol_desc& d = mols[m];
    if (d.norb < 1 || d.n < 2 || !(d.h > 0.0) || !std::isfinite(d.h) || !std::isfinite(d.alpha) ||
        d.occupations == nullptr || d.tile < 0)
      return EXX_ERR_INVALID_ARG;
    for (int i = 0; i < d.norb; ++i)
      if (!std::isfinite(d.occupations[i])) return EXX_ERR_INVALID_ARG;
    const Ops* ops = find_ops(EXX_FP32, d.n);
    if (ops == nullptr || !ops->supported) return EXX_ERR_NOT_SUPPORTED;
  }
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  exx_batch_t b = new exx_batch_s();
  b->nmol = nmol;
  b->kind = kernel;
  std::vector<double> occ;
  long long ep = 0, vo = 0;
  for (int m = 0; m < nmol; ++m) {
    const exx_mol_desc& d = mols[m];
    Mol mm;
    mm.n = d.n;
    mm.N = d.norb;
    mm.h = d.h;
    mm.alpha = d.alpha;
    mm.T = default_tile(d.norb, d.tile);
    mm.occ_off = (int)occ.size();
    occ.insert(occ.end(), d.occupations, d.occupations + d.norb);
    mm.P = (long long)d.norb * (d.norb + 1) / 2;
    mm.ep_off = ep;
    ep += mm.P;
    mm.vacc_off = vo;
    vo += (long long)d.norb * d.n * d.n * d.n;
    mm.group = -1;
    for (size_t g = 0; g < b->groups.size(); ++g)
      if (b->groups[g].n == d.n && b->groups[g].h == d.h) mm.group = (int)g;
    if (mm.group < 0) {
      Group g;
      g.n = d.n;
      g.h = d.h;
      g.kind = kernel;
      g.ops = find_ops(EXX_FP32, d.n);
      mm.group = (int)b->groups.size();
      b->groups.push_back(g);
    }
    b->groups[mm.group].mols.push_back(m);
    b->mol.push_back(mm);
  }
  // tiles of each molecule (row-major over blocks, as in a single plan), then
  // waves: round-robin over the group's molecules, one tile per molecule per
  // wave, up to the pair budget
  for (Group& g : b->groups) {
    std::vector<std::vector<TileDesc>> q(g.mols.size());
    std::vector<std::vector<std::vector<int4>>> qp(g.mols.size());
    for (size_t k = 0; k < g.mols.size(); ++k) {
      const Mol& m = b->mol[g.mols[k]];
      const int T = m.T, nb = (m.N + T - 1) / T;
      for (int bi = 0; bi < nb; ++bi)
        for (int bj = bi; bj < nb; ++bj) {
          TileDesc t;
          t.i0 = bi * T;
          t.ti = std::min(T, m.N - t.i0);
          t.j0 = bj * T;
          t.tj = std::min(T, m.N - t.j0);
          t.diag = bi == bj;
          t.mol = g.mols[k];
          t.occ_off = m.occ_off;
          t.c = -m.alpha;
          t.g2h3 = 2.0 * m.h * m.h * m.h;
          t.voff = 0;
          std::vector<int4> ps;
          for (int a = 0; a < t.ti; ++a)
            for (int c = t.diag ? a : 0; c < t.tj; ++c) {
              const int i = t.i0 + a, j = t.j0 + c;
              const long long gid = (long long)i * m.N - ((long long)i * (i - 1)) / 2 + (j - i);
              ps.push_back(make_int4(i, j, (int)(m.ep_off + gid), g.mols[k]));
            }
          q[k].push_back(t);
          qp[k].push_back(ps);
        }
    }
    std::vector<size_t> next(g.mols.size(), 0);
    for (;;) {
      Wave w;
      w.pair_off = (int)b->pairs.size();
      w.tile_off = (int)b->tiles.size();
      w.npair = 0;
      w.ntile = 0;
      for (size_t k = 0; k < g.mols.size(); ++k) {
        if (next[k] >= q[k].size()) continue;
        const std::vector<int4>& ps = qp[k][next[k]];
        if (w.npair > 0 && w.npair + (long long)ps.size() > kWavePairBudget) continue;
        TileDesc t = q[k][next[k]];
        t.voff = w.npair;
        b->tiles.push_back(t);
        b->pairs.insert(b->pairs.end(), ps.begin(), ps.end());
        w.npair += (int)ps.size();
        w.ntile += 1;
        next[k] += 1;
      }
      if (w.ntile == 0) break;
      g.waves.push_back(w);
      const size_t cs = sizeof(float2), rs = sizeof(float);
      const size_t n = (size_t)g.n;
      b->x_bytes = std::max(b->x_bytes, (size_t)w.npair * (n + 1) * n * 2 * n * cs);
      b->v_bytes = std::max(b->v_bytes, (size_t)w.npair * n * n * n * rs);
      b->ep_bytes = std::max(b->ep_bytes, (size_t)w.npair * (n + 1) * g.ops->nyb * sizeof(double));
      b->max_wave_pairs = std::max(b->max_wave_pairs, w.npair);
    }
  }
  // device data
  std::vector<MolTot> mt;
  std::vector<long long> count;
  for (const Mol& m : b->mol) {
    mt.push_back(MolTot{m.N, m.occ_off, m.ep_off, m.alpha});
    count.push_back((long long)m.N * m.n * m.n * m.n);
  }
  bool ok = balloc(b, &b->d_pairs, b->pairs.size() * sizeof(int4)) &&
            balloc(b, &b->d_tiles, b->tiles.size() * sizeof(TileDesc)) &&
            balloc(b, &b->d_occ, occ.size() * sizeof(double)) &&
            balloc(b, &b->Epair, (size_t)ep * sizeof(double)) && balloc(b, &b->epart, b->ep_bytes) &&
            balloc(b, &b->X, b->x_bytes) && balloc(b, &b->V, b->v_bytes) &&
            balloc(b, &b->vacc, (size_t)vo * sizeof(double)) &&
            balloc(b, &b->d_mt, mt.size() * sizeof(MolTot)) &&
            balloc(b, &b->d_psi_tab, nmol * sizeof(float*)) &&
            balloc(b, &b->d_vacc_tab, nmol * sizeof(double*)) &&
            balloc(b, &b->d_vx_tab, nmol * sizeof(float*)) &&
            balloc(b, &b->d_count, nmol * sizeof(long long));
  if (!ok) {
    batch_free(b);
    delete b;
    return EXX_ERR_OOM;
  }
  std::vector<double*> vtab;
  for (const Mol& m : b->mol) vtab.push_back(b->vacc + m.vacc_off);
  cudaError_t e = cudaSuccess;
  auto up = [&](void* dst, const void* src, size_t bytes) {
    if (e == cudaSuccess && bytes) e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st);
  };
  up(b->d_pairs, b->pairs.data(), b->pairs.size() * sizeof(int4));
  up(b->d_tiles, b->tiles.data(), b->tiles.size() * sizeof(TileDesc));
  up(b->d_occ, occ.data(), occ.size() * sizeof(double));
  up(b->d_mt, mt.data(), mt.size() * sizeof(MolTot));
  up(b->d_vacc_tab, vtab.data(), vtab.size() * sizeof(double*));
  up(b->d_count, count.data(), count.size() * sizeof(long long));
  if (e == cudaSuccess) e = cudaMemsetAsync(b->Epair, 0, (size_t)ep * sizeof(double), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->d_vx_tab, 0, nmol * sizeof(float*), st);
  // kernel spectra and twiddles per group
  for (Group& g : b->groups) {
    const size_t m = (size_t)g.n + 1;
    std::vector<double> Gh(m * m * m);
    if (!exx_host::kernel_spectrum_octant(g.n, g.h, kernel, 0.0, Gh.data())) {
      batch_free(b);
      delete b;
      return EXX_ERR_INVALID_ARG;
    }
    const double L = 2.0 * g.n, scale = 1.0 / (L * L * L);
    std::vector<double> gx(m), gy(2 * (size_t)g.n), gz(2 * (size_t)g.n);
    g.ops->gains(gx.data(), gy.data(), gz.data());
    std::vector<unsigned char> gf(exx::kernel_table_bytes(g.n, g.n, sizeof(float), g.ops->table_fold_y));
    exx::build_kernel_table<float>(g.n, g.n, g.ops->table_fold_y, Gh.data(), scale, gx.data(),
                                   gy.data(), gz.data(), gf.data());
    std::vector<float> tw(2 * exx::twiddle_count(g.n));
    exx::build_twiddles(g.n, tw.data());
    if (!balloc(b, &g.Gs, gf.size()) || !balloc(b, &g.tw, tw.size() * sizeof(float))) {
      batch_free(b);
      delete b;
      return EXX_ERR_OOM;
    }
    up(g.Gs, gf.data(), gf.size());
    up(g.tw, tw.data(), tw.size() * sizeof(float));
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // host buffers die at scope end
    if (e == cudaSuccess && g.ops->stage_table && !exx::make_ktab_map(&g.gmap, g.Gs, g.n, g.n))
      e = cudaErrorInvalidValue;
    if (e == cudaSuccess) e = g.ops->setup();
  }
  if (!balloc(b, &b->d_err, 2 * sizeof(int))) {
    batch_free(b);
    delete b;
    return EXX_ERR_OOM;
  }
  {
    size_t nwaves = 0;
    for (const Group& g : b->groups) nwaves += g.waves.size();
    const char* env = std::getenv("EXX_LANES");
    b->lanes = (env && env[0] == '1') || nwaves < 2 ? 1 : 2;
  }
  if (b->lanes > 1) {
    if (!balloc(b, &b->epart2, b->ep_bytes) || !balloc(b, &b->X_2, b->x_bytes) ||
        !balloc(b, &b->V_2, b->v_bytes)) {
      batch_free(b);
      delete b;
      return EXX_ERR_OOM;
    }
    for (int l = 0; l < 2 && e == cudaSuccess; ++l) {
      e = cudaStreamCreateWithFlags(&b->ls[l], cudaStreamNonBlocking);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_done[l], cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_free[l], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(b->d_err, 0, 2 * sizeof(int), st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    batch_free(b);
    delete b;
    return e == cudaErrorMemoryAllocation ? EXX_ERR_OOM : EXX_ERR_CUDA;
  }
  *out = b;
  return EXX_OK;
}

exx_status_t exx_batch_set_buffers(exx_batch_t b, const float* const* psi, float* const* vxpsi,
                                   void* cuda_stream) {
  if (b == nullptr || psi == nullptr) return EXX_ERR_INVALID_ARG;
  for (int m = 0; m < b->nmol; ++m)
    if (psi[m] == nullptr) return EXX_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  std::vector<const float*> p(psi, psi + b->nmol);
  std::vector<float*> v(b->nmol, nullptr);
  bool have = vxpsi != nullptr;
  if (have)
    for (int m = 0; m < b->nmol; ++m) {
      v[m] = vxpsi[m];
      if (v[m] == nullptr) have = false;
    }
  cudaError_t e = cudaMemcpyAsync(b->d_psi_tab, p.data(), b->nmol * sizeof(float*),
                                  cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->d_vx_tab, v.data(), b->nmol * sizeof(float*), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return EXX_ERR_CUDA;
  }
  bool v2 = true;
  for (int m = 0; m < b->nmol; ++m) v2 = v2 && ((uintptr_t)p[m] % 8 == 0);
  if (v2 != b->vec2 || have != b->have_vx) {  // the captured graphs embed these choices
    for (int k = 0; k < 3; ++k)
      if (b->gexec[k]) {
        cudaGraphExecDestroy(b->gexec[k]);
        b->gexec[k] = nullptr;
      }
  }
  b->vec2 = v2;
  b->have_vx = have;
  b->buffers_set = true;
  return EXX_OK;
}

exx_status_t exx_batch_apply(exx_batch_t b, double* E_dev, void* cuda_stream) {
  if (b == nullptr || E_dev == nullptr) return EXX_ERR_INVALID_ARG;
  return run_batch(b, E_dev, true, false, static_cast<cudaStream_t>(cuda_stream));
}

exx_status_t exx_batch_gradient(exx_batch_t b, double* E_dev, void* cuda_stream) {
  if (b == nullptr || E_dev == nullptr) return EXX_ERR_INVALID_ARG;
  return run_batch(b, E_dev, true, true, static_cast<cudaStream_t>(cuda_stream));
}

exx_status_t exx_batch_energy(exx_batch_t b, double* E_dev, void* cuda_stream) {
  if (b == nullptr || E_dev == nullptr) return EXX_ERR_INVALID_ARG;
  return run_batch(b, E_dev, false, false, static_cast<cudaStream_t>(cuda_stream));
}

exx_status_t exx_batch_set_persistent(exx_batch_t b, int enable, void* cuda_stream) {
  if (b == nullptr) return EXX_ERR_INVALID_ARG;
  if ((enable != 0) == b->persistent) return EXX_OK;
  for (int k = 0; k < 3; ++k)  // the captured graphs embed the schedule
    if (b->gexec[k]) {
      cudaGraphExecDestroy(b->gexec[k]);
      b->gexec[k] = nullptr;
    }
  if (!enable) {
    b->persistent = false;
    return EXX_OK;
  }
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  if (b->d_segs == nullptr) {
    const char* hook = std::getenv("EXX_TEST_STALL_QUEUE");
    const bool stall = hook != nullptr && hook[0] == '1';
    std::vector<QSeg> segs;
    int mx = 0;
    for (Group& g : b->groups)
      if (g.ops->persist_ok) {
        build_segments(b, g, true, stall, segs);
        build_segments(b, g, false, stall, segs);
        mx = std::max(mx, std::max(g.nseg[0], g.nseg[1]));
      }
    if (segs.empty()) return EXX_OK;  // no group has a persistent kernel
    // the queue reuses two workspace slots (those of the two pipeline lanes)
    if (b->X_2 == nullptr) {
      if (!balloc(b, &b->epart2, b->ep_bytes) || !balloc(b, &b->X_2, b->x_bytes) ||
          !balloc(b, &b->V_2, b->v_bytes))
        return EXX_ERR_OOM;
    }
    if (!balloc(b, &b->d_segs, segs.size() * sizeof(QSeg)) ||
        !balloc(b, &b->d_qc, (size_t)(mx + 2) * sizeof(int)))
      return EXX_ERR_OOM;
    b->qc_len = mx + 2;
    if (cudaMemcpyAsync(b->d_segs, segs.data(), segs.size() * sizeof(QSeg), cudaMemcpyHostToDevice,
                        st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      cudaGetLastError();
      return EXX_ERR_CUDA;
    }
    b->segs.swap(segs);
  }
  for (const Group& g : b->groups)  // function attributes and grid size, outside any capture
    if (g.ops->persist_ok) {
      PersistArgs none{};
      if (g.ops->persist(none, st) != cudaSuccess) {
        cudaGetLastError();
        return EXX_ERR_CUDA;
      }
    }
  b->persistent = true;
  return EXX_OK;
}

exx_status_t exx_batch_graph(exx_batch_t b, int enable) {
  if (b == nullptr) return EXX_ERR_INVALID_ARG;
  b->graph_on = enable != 0;
  return EXX_OK;
}

exx_status_t exx_batch_pair_energies(exx_batch_t b, int mol, double* out_host, void* cuda_stream) {
  if (b == nullptr || out_host == nullptr || mol < 0 || mol >= b->nmol) return EXX_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const Mol& m = b->mol[mol];
  int flag = 0;
  if (cudaMemcpyAsync(out_host, b->Epair + m.ep_off, (size_t)m.P * sizeof(double),
                      cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaMemcpyAsync(&flag, b->d_err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    cudaGetLastError();
    return EXX_ERR_CUDA;
  }
  if (flag) {  // a bounded device-side wait ran out
    cudaMemsetAsync(b->d_err, 0, sizeof(int), st);
    return EXX_ERR_TIMEOUT;
  }
  return EXX_OK;
}

exx_status_t exx_batch_info(exx_batch_t b, int* ngroups, int* nwaves, size_t* workspace_bytes,
                            int* launches_apply, long long* pairs) {
  if (b == nullptr) return EXX_ERR_INVALID_ARG;
  int nw = 0;
  for (const Group& g : b->groups) nw += (int)g.waves.size();
  if (ngroups) *ngroups = (int)b->groups.size();
  if (nwaves) *nwaves = nw;
  if (workspace_bytes) *workspace_bytes = b->ws;
  if (launches_apply) {
    int la = 2;  // E_x totals and the conversion of the outputs
    for (const Group& g : b->groups)
      la += (b->persistent && g.ops->persist_ok) ? 1 : 5 * (int)g.waves.size();
    *launches_apply = la;
  }
  if (pairs) *pairs = (long long)b->pairs.size();
  return EXX_OK;
}

exx_status_t exx_batch_destroy(exx_batch_t b) {
  if (b == nullptr) return EXX_OK;
  batch_free(b);
  delete b;
  return EXX_OK;
}

}  // extern "C"
