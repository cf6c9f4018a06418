/*
 * exx.h -- C ABI of the GB300 (sm_103a) exact-exchange operator.
 *
 * The library applies the exact-exchange (Fock) operator of hybrid density
 * functionals to N real orbitals sampled on a uniform cubic grid with free
 * (isolated) boundary conditions -- or, by kernel kind, periodic, slab or wire
 * cells -- following arXiv 1712.07973 (Ratcliff et al.):
 *
 *   rho_ij(r)  = psi_i(r) psi_j(r)                       (Sec. 2.1, kernel 1)
 *   V_ij       = G * rho_ij, the free-BC Poisson solution (Sec. 2.1.2, kernel 2;
 *                exact aperiodic convolution through a zero-padded 2n FFT)
 *   E_x        = -(alpha/2) sum_{i,j} f_i f_j h^3 sum_r rho_ij V_ij
 *                                                        (Sec. 2, Eq. HF and the
 *                                                         E_X equation after the
 *                                                         pair-count paragraph)
 *   (Vx psi)_i = -alpha sum_j f_j V_ij psi_j             (Sec. 2, Eq. daction)
 *
 * over all N(N+1)/2 pairs i <= j (Sec. 2, pair-count paragraph; Table
 * pscount), each pair feeding both i and j (Sec. 2.1, round-robin paragraph).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Orbital arrays are row-major [norb][n][n][n] with x fastest (index
 *   ((o*n + z)*n + y)*n + x), grid nodes at x_m = m*h, m = 0..n-1.
 * - "device" pointers are CUDA device (or managed) memory on the current
 *   device; "host" pointers are ordinary host memory.  The caller keeps
 *   ownership of every pointer it passes; the plan owns only what it allocates.
 * - cuda_stream is a cudaStream_t passed as void* (NULL = legacy default
 *   stream).  Work is enqueued on that stream; a plan with several pipeline
 *   lanes (exx_plan_set_lanes) forks onto internal streams after the work
 *   already on it and joins back before the call's last step, so the
 *   caller's stream order holds as if everything ran on it.
 * - Every entry point returns an exx_status_t and never aborts the process.
 *   On EXX_ERR_CUDA the CUDA error string is kept in the plan and returned by
 *   exx_last_error().
 * - A plan is not thread-safe: calls on one plan must not overlap in time
 *   (they share the plan's workspace).  Different plans are independent.
 */
#ifndef EXX_GB300_H
#define EXX_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct exx_plan_s* exx_plan_t;

typedef enum {
  EXX_OK = 0,
  EXX_ERR_INVALID_ARG = 1,   /* NULL pointer, n < 2, h <= 0, norb < 1, bad enum */
  EXX_ERR_CUDA = 2,          /* a CUDA runtime call failed (see exx_last_error)  */
  EXX_ERR_OOM = 3,           /* device workspace could not be allocated          */
  EXX_ERR_TIMEOUT = 4,       /* a bounded device-side wait gave up (reported by
                                the next synchronising call: exx_energy,
                                exx_apply with E_out, exx_apply_host,
                                exx_batch_pair_energies)                         */
  EXX_ERR_NOT_SUPPORTED = 5  /* non-cubic grid, 2n with a prime factor > 7, or a
                                size beyond the compiled kernels                  */
} exx_status_t;

typedef enum {
  EXX_FP64 = 0,  /* FFTs, products and reductions in FP64; psi/vxpsi are double  */
  EXX_FP32 = 1   /* FFTs and products in FP32, kernel built in FP64, E_x and the
                    Vx psi accumulation across pairs in FP64; psi is float        */
} exx_precision_t;

typedef enum {
  EXX_KERNEL_SINC = 0,    /* band-limited free-space kernel (default): exact for
                             densities band-limited to the grid's Brillouin zone */
  EXX_KERNEL_HOCKNEY = 1, /* point-sampled h^3/|r|, cell-averaged origin; O(h^2)  */
  EXX_KERNEL_ERFC = 2,    /* band-limited short-range kernel erfc(omega r)/r of
                             screened hybrids (HSE-type; Sec. 3 notes that only
                             the Poisson filter changes); needs omega > 0 and
                             exx_plan_create_desc                                 */
  EXX_KERNEL_PERIODIC = 3, /* periodic boundary conditions on the n^3 cell of side
                             n h (the paper's own runs, Sec. 3, are periodic):
                             V_hat = 4 pi rho_hat / |k|^2 with k = 0 removed, no
                             padding; n even, n in {8,12,16,24,32,48,64,96,128,
                             192}                                                 */
  EXX_KERNEL_SLAB = 4,    /* slab ("surface") boundary conditions (Sec. 2.1.2:
                             other boundary conditions change only the Green's
                             function): x and y periodic with the cell n h, z
                             free (zero-padded to 2n); per in-plane frequency k
                             the band-limited 1D kernel of d2/dz2 - k^2, at k = 0
                             the one whose potential of band-limited densities is
                             -2 pi int |z - z'| rho dz'; n in {8,16,32,48,64,96} */
  EXX_KERNEL_WIRE = 5     /* wire boundary conditions: x and y free (zero-padded),
                             z periodic with the cell n h; per axial frequency k
                             the band-limited 2D kernel of lap_2 - k^2, at k = 0
                             the one whose potential of band-limited densities is
                             -2 int ln|r - r'| rho d2r' (r in bohr);
                             n in {8,16,32,48,64,96}                              */
} exx_kernel_t;

/* Plan flags (bitwise or). */
#define EXX_FLAG_VX_FP64 1u  /* FP32 plans: write vxpsi as double instead of float */
/* Pair-tile edge T (1..8 orbitals per tile side) chosen by the caller, e.g. from
 * a tuning run; 0 (no flag) selects the default 8. */
#define EXX_FLAG_TILE(t) (((unsigned)(t) & 15u) << 8)

/*
 * exx_plan_create -- build a plan for fixed (grid, h, alpha, occupations).
 *   out          host, receives the plan handle (set to NULL on failure).
 *   grid[3]      host, points per axis (nx, ny, nz); must be equal (cubic),
 *                2 <= n, and 2n = 2^a 3^b 5^c 7^d within the compiled sizes.
 *   h[3]         host, grid spacing per axis in bohr; must be equal and > 0.
 *   alpha        exact-exchange fraction (PBE0: 0.25, Sec. 3).
 *   occupations  host, norb values f_i (Eq. 1); copied into the plan.
 *   norb         number of orbitals N >= 1.
 *   precision    exx_precision_t.
 *   kernel       exx_kernel_t.
 *   flags        EXX_FLAG_* bits.
 *   cuda_stream  stream for the plan's set-up uploads (synchronised on return).
 * The FP64 kernel spectrum is built on the host (Sec. 2.1.2 reading: the
 * Green's function discretised on the mesh), uploaded once, and workspaces for
 * one pair tile per pipeline lane are allocated with cudaMalloc.
 */
exx_status_t exx_plan_create(exx_plan_t* out, const int grid[3], const double h[3],
                             double alpha, const double* occupations, int norb,
                             int precision, int kernel, unsigned flags, void* cuda_stream);

/*
 * exx_plan_create_desc -- exx_plan_create with every option in one struct,
 * including the screening parameter omega (bohr^-1) of EXX_KERNEL_ERFC.
 */
typedef struct {
  int grid[3];
  double h[3];
  double alpha;
  const double* occupations;  /* host, norb values; copied */
  int norb;
  int precision;              /* exx_precision_t */
  int kernel;                 /* exx_kernel_t */
  unsigned flags;             /* EXX_FLAG_* */
  double omega;               /* EXX_KERNEL_ERFC only: erfc(omega r)/r, omega > 0 */
} exx_plan_desc;
exx_status_t exx_plan_create_desc(exx_plan_t* out, const exx_plan_desc* desc, void* cuda_stream);

/*
 * exx_energy -- E_x only (forward transforms and the Parseval sum; no inverse).
 *   psi    device, [norb][n][n][n], double (EXX_FP64) or float (EXX_FP32).
 *   E_out  host, receives E_x in hartree.  The call synchronises the stream.
 */
exx_status_t exx_energy(exx_plan_t plan, const void* psi, double* E_out, void* cuda_stream);

/*
 * exx_apply -- E_x and the exchange action vxpsi = (Vx psi)_i for all i.
 *   psi    device, as for exx_energy.
 *   vxpsi  device, [norb][n][n][n]; double for EXX_FP64 or with
 *          EXX_FLAG_VX_FP64, else float.  Overwritten (not accumulated).
 *   E_out  host, may be NULL.  If non-NULL the call synchronises the stream.
 * The gradient of E_x is dE_x/dpsi_k = 2 f_k h^3 (Vx psi)_k.
 */
exx_status_t exx_apply(exx_plan_t plan, const void* psi, void* vxpsi, double* E_out,
                       void* cuda_stream);

/*
 * exx_apply_async -- as exx_apply, but E_x is written to device memory and the
 * call never synchronises (E_dev: device, one double; may be NULL).
 */
exx_status_t exx_apply_async(exx_plan_t plan, const void* psi, void* vxpsi, double* E_dev,
                             void* cuda_stream);

/*
 * exx_gradient -- E_x and its gradient with respect to the orbitals,
 *   grad_k = dE_x/dpsi_k = 2 f_k h^3 (Vx psi)_k   (Sec. 2, Eq. daction: the
 *   Fock operator is the derivative of E_X with respect to the density
 *   matrix; for real orbitals and the symmetric kernel the factor 2 f_k h^3
 *   follows from rho_ij = psi_i psi_j and the h^3 quadrature),
 * from the same pair solves as exx_apply: the per-orbital factor is folded
 * into the FP64 accumulation, so no separate scaling pass is needed.
 *   psi    device, as for exx_energy.
 *   grad   device, same shape and dtype as exx_apply's vxpsi; overwritten.
 *   E_out  host, may be NULL; if non-NULL the call synchronises the stream.
 */
exx_status_t exx_gradient(exx_plan_t plan, const void* psi, void* grad, double* E_out,
                          void* cuda_stream);
/* exx_gradient_async -- as exx_gradient with E_x written to device memory
 * (E_dev: device, one double, may be NULL); never synchronises. */
exx_status_t exx_gradient_async(exx_plan_t plan, const void* psi, void* grad, double* E_dev,
                                void* cuda_stream);

/*
 * exx_energy_async -- as exx_energy with E_x written to device memory; no sync.
 */
exx_status_t exx_energy_async(exx_plan_t plan, const void* psi, double* E_dev,
                              void* cuda_stream);

/*
 * exx_pair_energies -- per-pair energies E_ij = h^3 sum_r rho_ij V_ij of the
 * last exx_energy/exx_apply call on this plan, copied to host memory in the
 * order (0,0),(0,1)..(0,N-1),(1,1),..,(N-1,N-1): N(N+1)/2 doubles.  Synchronises
 * the stream.
 */
exx_status_t exx_pair_energies(exx_plan_t plan, double* out_host, void* cuda_stream);

/*
 * exx_plan_info -- sizes chosen by the plan (host out-parameters, each may be
 * NULL): tile edge (orbitals per tile side), number of pair tiles, device
 * workspace bytes, number of kernel launches one exx_apply enqueues.
 */
exx_status_t exx_plan_info(exx_plan_t plan, int* tile, int* ntiles, size_t* workspace_bytes,
                           int* launches_apply, int* launches_energy);

/*
 * exx_apply_host -- exx_apply for callers whose orbitals live in host memory.
 *   psi_host    host, [norb][n][n][n] (double for EXX_FP64, float for EXX_FP32);
 *               page-locked memory gives asynchronous copies.
 *   vxpsi_host  host, same shape, dtype as for exx_apply; overwritten.
 *   E_out       host, may be NULL.
 * The first call allocates device buffers for psi and vxpsi inside the plan
 * (kept until exx_plan_destroy), a copy stream and events.  The call copies
 * psi in per block of T orbitals (the tile edge) on the copy stream, runs
 * exx_apply on the given stream with each tile waiting only for its two
 * blocks, copies each block of vxpsi out as soon as the last tile row that
 * touches it has finished (row-major tiles: block b after row b), copies E_x
 * out and synchronises both streams before returning.  Results equal those
 * of exx_apply bit for bit.  A sharded plan copies in one piece each way.
 */
exx_status_t exx_apply_host(exx_plan_t plan, const void* psi_host, void* vxpsi_host, double* E_out,
                            void* cuda_stream);
/* exx_gradient_host -- exx_apply_host returning the gradient 2 f_k h^3
 * (Vx psi)_k in grad_host (see exx_gradient); same buffers, overlap and
 * synchronisation. */
exx_status_t exx_gradient_host(exx_plan_t plan, const void* psi_host, void* grad_host,
                               double* E_out, void* cuda_stream);

/*
 * exx_plan_set_lanes -- number of pipeline lanes (1 to 3) of later calls.
 * A plan is created with two lanes, or one where its slab kernels run as
 * CTA clusters (FP32 n = 160, FP64 n >= 96), or EXX_LANES = 1, 2 or 3
 * from the environment at creation; never more than it has pair tiles; each beyond
 * the first with its own internal stream and spectrum and potential
 * workspaces.  Consecutive tiles go round-robin over the lanes, so the
 * transforms of one tile run beside those of the next; the accumulation stays
 * on the caller's stream in tile order and results are identical bit for bit.
 * One lane serialises every kernel on the caller's stream (per-kernel timing,
 * below, then measures each kernel alone).  Returns EXX_ERR_NOT_SUPPORTED for
 * more lanes than the plan was created with.
 */
exx_status_t exx_plan_set_lanes(exx_plan_t plan, int lanes);
/* exx_plan_get_lanes -- current number of lanes (host out-parameter). */
exx_status_t exx_plan_get_lanes(exx_plan_t plan, int* lanes);

/*
 * Per-kernel timing with CUDA events recorded on the launching stream around
 * every launch of the pipeline (kernel kinds, in order: 0 fwd_xy, 1 zconv,
 * 2 pair_energy, 3 inv_yx, 4 accum, 5 exx_total, 6 to_float).
 * exx_profile_enable(plan, 1) starts recording (0 stops); exx_profile_read
 * synchronises on the recorded events and returns, per kind, the summed
 * milliseconds (host ms[EXX_NKINDS]) and launch counts (host
 * launches[EXX_NKINDS]); reset != 0 clears the tallies afterwards.
 */
#define EXX_NKINDS 7
exx_status_t exx_profile_enable(exx_plan_t plan, int enable);
exx_status_t exx_profile_read(exx_plan_t plan, double* ms, long long* launches, int reset);

/*
 * exx_pair_energy_noalloc -- E_ij = h^3 sum_r rho_ij V_ij of one orbital pair
 * (FP32 path, same kernels as exx_energy) without a plan and without
 * allocating any device memory.  The paper has no counterpart: this entry
 * point exists for callers that cannot call cudaMalloc, such as codes that
 * give the whole device memory to their own pool allocator at start-up, or
 * that must keep allocation latency and its implicit synchronisation out of
 * their iteration loop.
 *   n, h, kernel   grid points per axis (2 <= n <= EXX_NOALLOC_MAX_N), spacing,
 *                  exx_kernel_t.
 *   psi            device, float [norb][n][n][n]; orbitals i and j are used.
 *   E_dev          device, one double, receives E_ij (no host copy, no sync);
 *                  NaN if a bounded device-side wait of the call ran out.
 * Scratch is a set of file-scope device arrays sized for EXX_NOALLOC_MAX_N
 * (about 29 MB, held by every GPU that loads the library until the process
 * exits).  n > EXX_NOALLOC_MAX_N returns EXX_ERR_NOT_SUPPORTED, as does a grid
 * without compiled kernels.  The first call on a device looks up the arrays'
 * device addresses (cudaGetSymbolAddress), and any call whose (n, h, kernel)
 * differs from the previous one on that device builds the kernel spectrum on
 * the host, copies it in and synchronises the stream: make such calls before
 * any stream capture.  That reload holds a per-device lock until the caller's
 * stream has drained, so calls on the same device from other host threads
 * wait meanwhile.  All calls on a device share the arrays, which keep the
 * last call's contents; calls that overlap on the GPU race and must be
 * serialised by the caller (one stream, or events).
 */
#define EXX_NOALLOC_MAX_N 96
exx_status_t exx_pair_energy_noalloc(int n, double h, int kernel, const float* psi, int norb,
                                     int i, int j, double* E_dev, void* cuda_stream);

/* ------------------------------------------------------------------------
 * Batched, uneven workloads: many independent molecules (each with its own
 * grid n, spacing, alpha, occupations and orbital count) in one call.
 * Molecules that share (n, h) share the kernel spectrum and every launch of
 * the pipeline; their pair tiles are scheduled in waves that take at most one
 * tile of each molecule, so each molecule's accumulation order, and result,
 * equals that of its own exx_plan with the same tile edge.  FP32 path only
 * (psi and vxpsi are float; kernel, energies and accumulation in FP64).
 * ------------------------------------------------------------------------ */
typedef struct exx_batch_s* exx_batch_t;

typedef struct {
  int n;                      /* grid points per axis (cubic)                  */
  double h;                   /* grid spacing, bohr                            */
  double alpha;               /* exact-exchange fraction                       */
  const double* occupations;  /* host, norb values; copied at creation         */
  int norb;                   /* orbitals                                      */
  int tile;                   /* pair-tile edge 1..8 (0: default 8)            */
} exx_mol_desc;

/*
 * exx_batch_create -- plan a batch of nmol molecules (mols: host array).
 * kernel: exx_kernel_t.  Allocates the workspace of the largest wave (waves
 * hold at most 512 pair solves) and one FP64 accumulator per molecule.
 */
exx_status_t exx_batch_create(exx_batch_t* out, int nmol, const exx_mol_desc* mols, int kernel,
                              void* cuda_stream);

/*
 * exx_batch_set_buffers -- bind the orbital and output arrays: psi, vxpsi are
 * host arrays of nmol device pointers (float [norb_m][n_m]^3 each); vxpsi may
 * be NULL for energy-only use.  The pointers are copied into device tables
 * that later calls (and captured graphs) read, so rebinding does not require
 * a new capture.  Synchronises the stream.
 */
exx_status_t exx_batch_set_buffers(exx_batch_t batch, const float* const* psi,
                                   float* const* vxpsi, void* cuda_stream);

/*
 * exx_batch_apply / exx_batch_energy -- E_x of every molecule into E_dev
 * (device, nmol doubles) and, for apply, Vx psi into the bound outputs.
 * Asynchronous on the stream.
 */
exx_status_t exx_batch_apply(exx_batch_t batch, double* E_dev, void* cuda_stream);
exx_status_t exx_batch_energy(exx_batch_t batch, double* E_dev, void* cuda_stream);
/*
 * exx_batch_gradient -- as exx_batch_apply, but the bound outputs receive the
 * gradient 2 f_k h^3 (Vx psi)_k of each molecule's E_x (see exx_gradient).
 */
exx_status_t exx_batch_gradient(exx_batch_t batch, double* E_dev, void* cuda_stream);

/*
 * exx_batch_graph -- enable (1) or disable (0) CUDA-graph execution: the next
 * apply (or energy) call captures its whole enqueue sequence on the given
 * stream (which must be a created stream, not the legacy default stream) and
 * launches the graph; later calls with the same stream and E_dev relaunch it.
 */
exx_status_t exx_batch_graph(exx_batch_t batch, int enable);

/*
 * exx_batch_set_persistent -- enable (1) or disable (0) the persistent
 * schedule: each group of molecules with the same (n, h) runs as ONE launch of
 * a persistent kernel that takes the (wave, pass, unit) items of all its pair
 * tiles from a device work queue, instead of five launches per wave.  Items of
 * a pass wait (bounded, on the device) for the items they depend on: a wait
 * that runs out sets the flag that exx_batch_pair_energies reports as
 * EXX_ERR_TIMEOUT, and the rest of the launch is skipped.  Results equal those
 * of the launch-per-pass schedule bit for bit.  FP32 grids whose slab kernels
 * run as CTA clusters (n = 160) keep the launch-per-pass schedule.  The first
 * enable builds the queue tables, allocates a second workspace slot if the
 * batch has none (returns EXX_ERR_OOM if that fails) and synchronises the
 * stream; it discards captured graphs.
 */
exx_status_t exx_batch_set_persistent(exx_batch_t batch, int enable, void* cuda_stream);

/* exx_batch_pair_energies -- pair energies of molecule mol (order as in
 * exx_pair_energies) of the last call, to host memory; synchronises. */
exx_status_t exx_batch_pair_energies(exx_batch_t batch, int mol, double* out_host,
                                     void* cuda_stream);

/* exx_batch_info -- (n, h) groups, waves, device workspace bytes, kernel
 * launches of one apply, total pair solves (each out-parameter may be NULL). */
exx_status_t exx_batch_info(exx_batch_t batch, int* ngroups, int* nwaves, size_t* workspace_bytes,
                            int* launches_apply, long long* pairs);

/* exx_batch_destroy -- free the batch (NULL is a no-op). */
exx_status_t exx_batch_destroy(exx_batch_t batch);

/*
 * Sharding over ranks (one GPU per rank).  Pair solves are independent, so a
 * rank can own a subset of the pair tiles; the only exchange is the sum of
 * E_x and of Vx psi over ranks (an all-reduce the caller performs, e.g. with
 * NCCL).  Tiles are assigned largest-first to the least-loaded rank (ties to
 * the lowest rank), which is deterministic and balances pair solves within one
 * tile.
 *
 * exx_shard_tiles -- host-only: the tile table of a plan with (norb, tile)
 *   and each tile's owner among nranks.  desc_out: host, 5 ints per tile
 *   (i0, ti, j0, tj, diag) in the plan's order; owner_out: host, one int per
 *   tile; either may be NULL to query *ntiles only.  Needs no GPU.
 * exx_plan_set_shard -- restrict the plan to the tiles of rank `rank` of
 *   `nranks` (1 rank = everything).  exx_energy / exx_apply then return this
 *   rank's partial E_x and partial Vx psi; summing them over ranks gives the
 *   full result.
 */
exx_status_t exx_shard_tiles(int norb, int tile, int nranks, int* desc_out, int* owner_out,
                             int* ntiles);
exx_status_t exx_plan_set_shard(exx_plan_t plan, int rank, int nranks);

/* exx_plan_destroy -- free the plan and its device memory (NULL is a no-op). */
exx_status_t exx_plan_destroy(exx_plan_t plan);

/*
 * exx_kernel_spectrum -- host-only: the FP64 spectrum of the zero-padded mesh
 * kernel, Ghat[k] = sum_d G~[d] exp(-i pi k.d / n) for k in [0, n]^3 (one
 * octant; Ghat is real and even per axis), unscaled.  omega is used by
 * EXX_KERNEL_ERFC only.  out_host holds (n+1)^3 doubles, index
 * (kz*(n+1) + ky)*(n+1) + kx.  EXX_KERNEL_PERIODIC (n even): 4 pi / |k|^2,
 * k = 2 pi m / (n h), m in [0, n/2]^3, 0 at m = 0; (n/2+1)^3 doubles.
 * EXX_KERNEL_SLAB (n even): kz in [0, n] (padded axis), kx, ky in [0, n/2];
 * (n+1)(n/2+1)^2 doubles, index (kz*(n/2+1) + ky)*(n/2+1) + kx.
 * EXX_KERNEL_WIRE (n even): kz in [0, n/2] (periodic axis), kx, ky in [0, n];
 * (n/2+1)(n+1)^2 doubles, index (kz*(n+1) + ky)*(n+1) + kx.
 * Needs no GPU.
 */
exx_status_t exx_kernel_spectrum(int n, double h, int kernel, double omega, double* out_host);

/* exx_status_string -- static text for a status code. */
const char* exx_status_string(exx_status_t status);

/* exx_last_error -- text of the last CUDA failure seen by this plan (or ""). */
const char* exx_last_error(exx_plan_t plan);

/* exx_version -- library version string. */
const char* exx_version(void);

#ifdef __cplusplus
}
#endif

#endif /* EXX_GB300_H */
