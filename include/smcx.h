/*
 * smcx.h -- C ABI of the GB300 SMC-X swap-sweep library (libsmcx.so).
 *
 * The library runs the hot path of SMC-X (arXiv 2509.20949) with the EPI
 * model: Metropolis swap trials (Sec. 2.1, Eq. 3) over a checkerboard of
 * link cells whose origin moves every MC step (Sec. 2.2, Eq. 5), each trial's
 * energy change taken from the local interaction zone of the swapped pair
 * (Sec. 2.2) with pairwise shell interactions only (Sec. 3, EPI model), plus
 * the Warren-Cowley short-range order (Sec. 3.2, Eq. 9) and the total energy.
 *
 * Conventions shared by every call:
 *  - Every function returns an smcx_status; nothing throws or longjmps across
 *    the ABI.  On failure smcx_last_error() (per host thread) describes why.
 *    Errors of a call that ran on the GPU (SMCX_ECUDA, SMCX_ETIMEOUT) are
 *    sticky on the handle: later calls return SMCX_ESTATE until destroy.
 *  - Memory ownership: the caller owns every device buffer (occupancy,
 *    workspace) and the CUDA stream; the library keeps non-owning pointers
 *    and never calls cudaMalloc/cudaFree.  Host pointers are only read or
 *    written during the call.
 *  - Canonical occupancy layout (what crosses the ABI on the host side): one
 *    byte per site holding the species id in [0, K), site index
 *    ((z*n_y + y)*n_x + x)*nb + b, nb = 2 (BCC basis (0,0,0),(1,1,1)) or
 *    4 (FCC basis (0,0,0),(0,1,1),(1,0,1),(1,1,0)), positions in half units
 *    2*(x,y,z) + basis.  The lattice is periodic in all three directions.
 *  - Energies are int64 in units of q = 2^-32 eV.  EPI tables are
 *    [n_shells][K][K] int64, symmetric, shells in ascending distance
 *    (BCC squared lengths 3,4,8,11; FCC 2,4,6,8 in (a/2)^2).
 *  - Stream order: calls enqueue on the handle's stream; calls that return
 *    host-visible results synchronise that stream before returning.
 *  - One handle is used by one host thread at a time.
 */
#ifndef SMCX_H
#define SMCX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SMCX_OK = 0,
  SMCX_EINVAL = 1,    /* bad argument: sizes, species id >= K, asymmetric V, ... */
  SMCX_ENOMEM = 2,    /* a caller buffer is too small */
  SMCX_ECUDA = 3,     /* a CUDA runtime call or kernel failed */
  SMCX_EOVERFLOW = 4, /* an energy total does not fit int64 */
  SMCX_ETIMEOUT = 5,  /* a bounded device-side wait gave up */
  SMCX_ESTATE = 6,    /* call not valid in the handle's state (no EPI yet, sticky error) */
  SMCX_EBUDGET = 7    /* batch admission refused: memory budget or slots exhausted */
} smcx_status;

#define SMCX_BCC 0u
#define SMCX_FCC 1u

/* smcx_lattice_desc.flags */
#define SMCX_NO_SHIFT 1u     /* keep the link-cell origin fixed (no per-step shift) */
#define SMCX_SINGLE_CELL 2u  /* one link cell: fully sequential sweeps (tiny lattices) */

typedef struct smcx_lattice smcx_lattice; /* opaque handle */

typedef struct {
  uint32_t kind;      /* SMCX_BCC or SMCX_FCC */
  uint32_t n[3];      /* conventional cells per dimension (periodic), each >= 1 */
  uint32_t n_species; /* K: 1..255 (1..16 when pack_bits == 4) */
  uint32_t pack_bits; /* device storage: 8 (one byte per site) or 4 (two sites per byte) */
  uint32_t min_cell;  /* link-cell edge floor in conventional cells; 0 = smallest safe edge */
  uint32_t flags;     /* SMCX_NO_SHIFT | SMCX_SINGLE_CELL */
  uint64_t seed;      /* Philox key (low word, high word) */
} smcx_lattice_desc;

typedef struct {
  uint64_t attempts; /* trials made (one per site per sweep, Sec. 2.1) */
  uint64_t unlike;   /* trials whose two sites held different species */
  uint64_t accepted; /* accepted swaps */
  int64_t sum_dE_q;  /* sum of the accepted energy changes (q units) */
} smcx_sweep_stats;

/* ---- sizes --------------------------------------------------------------- */

/* Device bytes the caller must provide for the occupancy (rounded up to 16).
   Returns 0 for an invalid descriptor. */
size_t smcx_occupancy_bytes(const smcx_lattice_desc* desc);

/* Device bytes the caller must provide as workspace (counters, EPI tables,
   pair-count accumulators).  Returns 0 for an invalid descriptor. */
size_t smcx_workspace_bytes(const smcx_lattice_desc* desc);

/* ---- lattice life cycle ------------------------------------------------- */

/* Validates desc and h_init (N = nb*n_x*n_y*n_z bytes, canonical layout,
   every id < K), binds the caller's device buffers d_occ
   (smcx_occupancy_bytes) and d_work (smcx_workspace_bytes, 256-byte
   aligned) and the stream (a cudaStream_t, NULL = legacy default stream),
   uploads the configuration and sets the sweep counter to 0.  No EPI is set
   yet.  *out receives the handle.  EINVAL: bad descriptor, N >= 2^32,
   species id >= K, misaligned buffers.  ECUDA: upload failed. */
smcx_status smcx_create_lattice(const smcx_lattice_desc* desc, void* d_occ, void* d_work,
                                const uint8_t* h_init, void* cuda_stream, smcx_lattice** out);

/* Sets the EPI model (Sec. 3: pairwise only): v_q is [n_shells][K][K] int64
   in q units, symmetric in the species indices; n_shells in 1..4.  The link
   cells are sized from the shells (edge L = floor((1 + h_R)/2) + 1
   conventional cells, h_R the largest |component| of a shell vector, raised
   to min_cell).  Restarts the running energy (see smcx_running_energy),
   which runs one pair count.  EINVAL: n_shells out of range, asymmetric V
   or a value beyond 2^52 q.  EOVERFLOW: the energy of the current
   configuration does not fit int64. */
smcx_status smcx_set_epi(smcx_lattice* lat, uint32_t n_shells, const int64_t* v_q);

/* Runs n_sweeps MC steps (one trial per site each, Sec. 2.1) on the stream.
   Sweep i of the call (0-based) runs at T_i = T_first + (T_last - T_first)
   * i / (n_sweeps - 1) kelvin (T_first when n_sweeps == 1 or T_first ==
   T_last); T = +inf accepts every unlike proposal, T = 0 accepts only
   dE <= 0.  Trial k of cell c in global sweep t uses Philox4x32-10 counter
   (k >> 1, c, t, 0) under the seed.  Advances the sweep counter by
   n_sweeps.  *out (host, may be NULL) receives the call's totals; when it is
   non-NULL the call synchronises the stream.  ESTATE: no EPI.  EINVAL: T < 0
   or NaN. */
smcx_status smcx_sweep(smcx_lattice* lat, uint32_t n_sweeps, double T_first, double T_last,
                       smcx_sweep_stats* out);

/* Runs the trials of one colour (0..7) of the current sweep (the sweep
   counter is not advanced) at temperature T.  Lets a caller replay and check
   single checkerboard phases; a full smcx_sweep runs colours 0..7 in order.
   Synchronises the stream when out != NULL. */
smcx_status smcx_run_colour(smcx_lattice* lat, uint32_t colour, double T, smcx_sweep_stats* out);

/* Full energy recomputed from the current occupancy (directed pair counts on
   the GPU, int128 sum on the host).  Synchronises.  EOVERFLOW if it does not
   fit int64.  ESTATE: no EPI. */
smcx_status smcx_energy(smcx_lattice* lat, int64_t* e_q);

/* Running energy: E_0 + the exact sum of every energy change accepted since
   the last restart.  E_0 is the full energy (a pair count) taken AT the
   restart -- smcx_set_epi, smcx_set_local_model, smcx_set_occupancy -- or
   the running energy stored in the checkpoint by smcx_restore, so comparing
   it with smcx_energy later checks the incremental bookkeeping against a
   recompute.  Only reads the device sum.  Synchronises.  ESTATE: no model
   set. */
smcx_status smcx_running_energy(smcx_lattice* lat, int64_t* e_q);

/* Warren-Cowley SRO, Sec. 3.2, Eq. 9.  pair_counts (host, required) receives
   [n_shells][K][K] uint64 directed counts N_m[p'][p] = number of (centre of
   species p', shell-m neighbour of species p) pairs over every site.
   alpha (host, may be NULL) receives alpha_m^{p p'} = 1 - N_m[p'][p] N /
   (N_{p'} z_m N_p) at [m][p'][p], NaN where a species is absent.
   n_shells 1..4 (independent of the EPI).  Synchronises. */
smcx_status smcx_warren_cowley_sro(smcx_lattice* lat, uint32_t n_shells, uint64_t* pair_counts,
                                   double* alpha);

/* Copies the occupancy to h_out (N bytes, canonical layout).  Synchronises. */
smcx_status smcx_get_occupancy(smcx_lattice* lat, uint8_t* h_out);

/* Starts copying the occupancy as it is now to h_out (N bytes, canonical
   layout; the caller keeps it alive, pinned host memory makes the copy
   asynchronous and fast) and returns without waiting.  The conversion to
   the canonical layout is enqueued on the lattice's stream, so the copy
   holds the occupancy of this point of the stream; the device-to-host copy
   itself runs on a copy stream of the handle and overlaps the calls that
   follow (a pair count, a sweep).  h_out is complete after
   smcx_wait_occupancy.  Calls that use the handle's transfer buffer
   (occupancy uploads and downloads, the composition profile) are ordered
   after the copy on the device.  Starting another asynchronous copy before
   waiting is allowed; smcx_wait_occupancy then waits for the last one. */
smcx_status smcx_get_occupancy_async(smcx_lattice* lat, uint8_t* h_out);

/* Waits until the copy started by the last smcx_get_occupancy_async has
   reached the host (returns at once when there is none). */
smcx_status smcx_wait_occupancy(smcx_lattice* lat);

/* Replaces the occupancy by h_in (N bytes, canonical, ids < K, validated on
   the device; on EINVAL the occupancy is left as it was) and restarts the
   running energy (one pair count once a model is set).  The sweep counter
   is unchanged.  Synchronises. */
smcx_status smcx_set_occupancy(smcx_lattice* lat, const uint8_t* h_in);

/* Composition profile along a cylinder (the atom-probe-like analysis of
   Sec. 3.2, whose cylinders are r = 12a, l = 72a): positions in half units
   h = a/2 (site 2*(x,y,z) + basis).  The cylinder's axis is lattice axis
   `axis` (0 = x, 1 = y, 2 = z) through origin_h[3]; a site at h is inside
   when t = (h_axis - origin_axis) mod 2n_axis < length_h and the squared
   minimum-image distance to the axis (each other component taken in
   (-n_d, n_d] modulo 2n_d) is <= radius2_h.  counts[bin][K] (host, n_bins
   x K) receives the species counts per bin, bin = t * n_bins / length_h.
   EINVAL: axis > 2, length_h outside 1..2n_axis, n_bins = 0, n_bins * K >
   8192 or 8 n_bins K > sites.  Synchronises. */
smcx_status smcx_composition_profile(smcx_lattice* lat, uint32_t axis, const int32_t* origin_h,
                                     uint64_t radius2_h, uint32_t length_h, uint32_t n_bins,
                                     uint64_t* counts);

/* Clusters (precipitates, Sec. 3.2): connected components of the sites whose
   species s has bit s set in species_mask, two such sites being connected
   when they are first-shell neighbours (periodic).  d_scratch: caller's
   device buffer of >= 8 bytes per site, 16-byte aligned (contents
   overwritten).  *n_clusters = number of clusters; sizes[0..min(cap,
   n_clusters)) (host) = the largest cluster sizes in descending order.
   ETIMEOUT: a capped device loop gave up (the handle then stays in error).
   Synchronises. */
smcx_status smcx_clusters(smcx_lattice* lat, uint32_t species_mask, void* d_scratch,
                          size_t scratch_bytes, uint64_t* n_clusters, uint64_t* sizes,
                          uint64_t cap);

/* Sweep counter (the global sweep index t of the next sweep). */
smcx_status smcx_get_sweep_counter(smcx_lattice* lat, uint32_t* t);
smcx_status smcx_set_sweep_counter(smcx_lattice* lat, uint32_t t);

/* Link-cell geometry chosen for the current EPI: edge L (conventional cells)
   and cells per dimension m[3] (even, or 1). ESTATE: no EPI. */
smcx_status smcx_get_layout(smcx_lattice* lat, uint32_t* L, uint32_t* m);

/* ---- local-energy model (the nonlinear short-range model of Sec. 3) -------
 *
 * The paper's second model (qSRO) is a general nonlinear short-range model: a
 * trial's energy change comes from recomputing the local energy of every
 * site in its interaction zone.  The paper does not print its functional
 * form; this library reads it as per-site energies that are tabulated
 * functions of the site's shell-resolved species counts:
 *   E = sum_i eps(i),  eps(i) = sum_m sum_s T_m[s_i][s][c_{i,m,s}],
 * c_{i,m,s} = the number of shell-m neighbours of i holding species s (each
 * shell displacement counted).  Any function of each count can be tabulated
 * (EPI is the linear case T_m[a][s][c] = c V_m(a, s) / 2).  A swap of i and j
 * changes eps only on U = {i, j} u shells(i) u shells(j); the kernel
 * recomputes eps before and after the swap on every distinct site of U.  A
 * trial then reads up to 1 + 2 h_R half units from its cell, so the link
 * cells grow to edge floor((1 + 2 h_R)/2) + 1.  The trial schedule, random
 * numbers and Metropolis test are those of the EPI sweep. */

/* Length zt of the count axis of a local-energy table: 1 + the largest
   coordination number of shells 1..n_shells.  0 for kind > 1 or n_shells
   outside 1..3. */
uint32_t smcx_local_model_width(uint32_t kind, uint32_t n_shells);

/* Replaces the lattice's energy model by the local-energy model with table
   t_q: [n_shells][K][K][zt] int64 q units (host, read during the call),
   entry [m][a][s][c] = the energy of a site of species a whose shell m+1
   holds c sites of species s.  Every later smcx_sweep / smcx_run_colour /
   smcx_energy / smcx_running_energy uses it (the SRO pair counts do not
   depend on the model); smcx_set_epi switches back.  Restarts the running
   energy.  EINVAL: n_shells outside 1..3, K > 8, some n_d < 4, or a table
   value beyond 2^48 in magnitude.  Checkpoints hold EPI lattices only
   (smcx_checkpoint returns ESTATE under this model), and the z
   decomposition plans are for EPI link cells. */
smcx_status smcx_set_local_model(smcx_lattice* lat, uint32_t n_shells, const int64_t* t_q);

/* ---- lattice decomposition along z (Sec. 2.2, lattice parallelism) -------
 *
 * The paper splits one lattice over several GPUs, each sweeping its own part
 * and trading boundary layers ("ghost layers") with its neighbours.  Here the
 * split is along z, in whole link-cell planes of each sweep's moving grid, and
 * it reproduces the single-lattice trajectory bit for bit:
 *  - in sweep t, rank r of R sweeps the link cells whose z index c lies in
 *    [floor(r m_z / R), floor((r+1) m_z / R)) (m_z >= 2R: two planes or more
 *    each); those cells cover conventional z planes
 *    [z_lo, z_lo + n_own) mod n_z, z_lo = s_z + floor(c_lo n_z / m_z) with
 *    the sweep's origin shift s_z;
 *  - every rank keeps the whole lattice (one byte per site fits many
 *    billions of sites in HBM) but its copy is only current on its window
 *    [z_lo - halo, z_lo + n_own + halo), halo = the link-cell edge L, which
 *    covers every site its trials read or write;
 *  - colours 0-3 are the even cell planes and 4-7 the odd ones.  Two cells
 *    of one z parity never interact, so during a half sweep (colours 0-3,
 *    then 4-7) no site one rank reads is written by another, and a site is
 *    written by at most one rank.  After each half sweep the two ranks on
 *    either side of an ownership boundary trade the 2 halo planes around it
 *    and merge them as mine ^ theirs ^ (the planes before the half sweep);
 *  - when the grid moves for sweep t + 1, each rank fetches the planes of its
 *    new window from their owners in sweep t (smcx_slab_transfer).
 * The per-rank statistics add up to the single-lattice ones. */

typedef struct {
  int32_t c_lo, c_hi; /* link-cell z indices [c_lo, c_hi) this rank sweeps */
  int32_t z_lo;       /* first owned conventional z plane, 0 <= z_lo < n_z */
  int32_t n_own;      /* owned planes z_lo .. z_lo + n_own - 1 (mod n_z) */
  int32_t halo;       /* planes on each side of an ownership boundary (= L) */
  int32_t m_z;        /* link cells along z */
} smcx_slab;

/* Plan of rank `rank` of `world` in sweep t for a lattice with this
   descriptor and an EPI of n_shells shells (pure host arithmetic: no handle,
   no GPU).  EINVAL: bad descriptor, n_shells outside 1..4, world = 0,
   rank >= world, or world > 1 with m_z < 2 world. */
smcx_status smcx_slab_plan(const smcx_lattice_desc* desc, uint32_t n_shells, uint32_t world,
                           uint32_t rank, uint32_t t, smcx_slab* out);

/* Planes that rank `from` owned in sweep t and rank `to` reads in sweep t+1
   (its window): *n_runs (0..2) runs (z0, nz), z0 in [0, n_z), written to
   runs[2 * i], runs[2 * i + 1] (host, room for 4 int32).  from == to gives
   0 runs.  Errors as smcx_slab_plan. */
smcx_status smcx_slab_transfer(const smcx_lattice_desc* desc, uint32_t n_shells, uint32_t world,
                               uint32_t from, uint32_t to, uint32_t t, int32_t* runs,
                               uint32_t* n_runs);

/* Runs colour `colour` (0..7) of the current sweep at temperature T on the
   link cells whose z index lies in [c_lo, c_hi) only (0 <= c_lo <= c_hi <=
   m_z); the sweep counter is not advanced.  A rank of a decomposition runs
   colours 4h .. 4h+3 on its [c_lo, c_hi) for half sweep h.  The call's
   statistics count those cells only (and add to the running energy).
   Synchronises the stream when out != NULL.  ESTATE: no EPI. */
smcx_status smcx_run_colour_planes(smcx_lattice* lat, uint32_t colour, double T, int32_t c_lo,
                                   int32_t c_hi, smcx_sweep_stats* out);

/* Device bytes of nz conventional z planes in device storage order (all
   basis rows of those planes: groups x nz x n_y x row pitch). */
size_t smcx_planes_bytes(smcx_lattice* lat, uint32_t nz);

/* Device-to-device copies, enqueued on the lattice's stream, between the
   planes z0 .. z0 + nz - 1 (mod n_z; nz <= n_z) of the occupancy and a
   caller's device buffer of smcx_planes_bytes(lat, nz) bytes (16-byte
   aligned): get reads the lattice, put overwrites it.  EINVAL: bad range,
   null or misaligned buffer. */
smcx_status smcx_get_planes(smcx_lattice* lat, int32_t z0, uint32_t nz, void* d_dst);
smcx_status smcx_put_planes(smcx_lattice* lat, int32_t z0, uint32_t nz, const void* d_src);

/* Merges another rank's copy of planes z0 .. z0 + nz - 1 into the lattice:
   occupancy ^= d_theirs ^ d_before, bytewise, where d_before holds the
   planes as both ranks had them before the half sweep (each site changed on
   at most one side).  Device buffers as smcx_get_planes; kernel on the
   lattice's stream. */
smcx_status smcx_merge_planes(smcx_lattice* lat, int32_t z0, uint32_t nz, const void* d_theirs,
                              const void* d_before);

/* Checkpoint: a self-describing byte string (descriptor, EPI, sweep counter,
   running energy, occupancy, CRC-32).  With buf == NULL, *len receives the
   size needed; otherwise *len must be at least that size and receives the
   bytes written.  ENOMEM: buffer too small.  Synchronises. */
smcx_status smcx_checkpoint(smcx_lattice* lat, void* buf, size_t* len);

/* Restores a checkpoint written by smcx_checkpoint for a lattice with the
   same descriptor.  EINVAL: wrong size, descriptor mismatch or CRC failure
   (the handle is left unchanged). */
smcx_status smcx_restore(smcx_lattice* lat, const void* buf, size_t len);

/* Tuning knobs (do not change results, only speed):
     SMCX_OPT_KERNEL   0 = automatic (tuned online: the first colour phases of
                       smcx_sweep rotate over the kernels and tile shapes
                       that can run the lattice, each timed with CUDA events
                       three times, and the fastest is kept; until then the
                       tiled kernel, else cell, else generic),
                       1 = generic (global memory, any lattice),
                       2 = tiled (shared-memory tiles + halos, large lattices),
                       3 = cell (one thread per link cell, n_d >= 4)
                       (a sweep fails with EINVAL if the requested kernel
                       cannot run the lattice).  Under the local-energy
                       model every sweep runs its own kernel, reported as 4
                       by smcx_kernel_in_use, whatever this option says
     SMCX_OPT_TILE     index of the tile shape among smcx_tile_shape(...)
     SMCX_OPT_STAGING  how the tiled kernel fills its shared-memory tiles:
                       0 = one bulk (TMA) copy per tile row wherever the
                       row's 16-byte aligned span fits (default), 8-byte
                       cp.async copies elsewhere; 1 = 8-byte cp.async copies
                       only */
#define SMCX_OPT_KERNEL 1u
#define SMCX_OPT_TILE 2u
#define SMCX_OPT_STAGING 3u
smcx_status smcx_set_option(smcx_lattice* lat, uint32_t key, int64_t value);

/* Number of tile shapes compiled for a lattice kind and the cells per tile
   (x, y, z) of shape i. */
uint32_t smcx_tile_shape_count(uint32_t kind);
smcx_status smcx_tile_shape(uint32_t kind, uint32_t i, uint32_t* cells_xyz);

/* Kernel the next sweep will use for this lattice and EPI: *kernel = 1
   (generic), 2 (tiled) or 3 (cell), 0 if the requested kernel cannot run
   it, and *tile_shape = the tile shape index (-1 unless tiled).
   ESTATE: no EPI. */
smcx_status smcx_kernel_in_use(smcx_lattice* lat, uint32_t* kernel, int32_t* tile_shape);

/* State of the online kernel choice: *done = 1 once decided; on entry
   *n_candidates = capacity of the arrays (may be 0 and the arrays NULL), on
   return the number of candidates; kernels[c] (1 generic, 2 tiled, 3 cell),
   shapes[c] (tile shape, -1 unless tiled) and best_ms[c] (fastest timed
   phase, -1 if not timed yet), each array may be NULL.  ESTATE: no EPI. */
smcx_status smcx_kernel_tuning(smcx_lattice* lat, uint32_t* done, uint32_t* n_candidates,
                               uint32_t* kernels, int32_t* shapes, float* best_ms);

/* Releases the handle (never the caller's buffers). */
smcx_status smcx_destroy(smcx_lattice* lat);

/* Text of the last error of this host thread ("" if none). */
const char* smcx_last_error(void);

/* ---- batched execution ---------------------------------------------------
   Many independent lattices (the paper's temperature parallelism, Sec. 2.2:
   simulations at different temperatures or compositions share nothing) run
   together.  Work items are 32 active link cells of one job and colour
   phase, one per lane of a warp.  Two schedules: a chunk of sweeps of all
   active jobs as one cooperative launch of a persistent kernel following a
   plan built on the host -- every warp owns fixed ranges of items of some
   jobs, the same in every colour phase, the jobs with the longest chains of
   dependent trials spread first -- with a per-job counter of finished items
   keeping each job's colour phases in sequence (bounded waits: a wait that
   gives up fails the run with ETIMEOUT); or one launch per colour phase
   covering all jobs.  The schedule, item shape and register budget are tuned online.
   With a stream the chunk is captured into a CUDA graph.  Each job's trajectory is
   bit-identical to the same lattice run alone through smcx_sweep (same
   seed, temperature and sweep counter), whatever the tuning.  Jobs use 8-bit
   storage, K <= 6, 2..4 shells, n >= 4 per dimension, a constant
   temperature.

   Memory: the caller provides one device arena (256-byte aligned); its first
   smcx_batch_control_bytes(max_jobs, transfer_bytes) bytes hold tables and
   two transfer buffers of transfer_bytes (>= the largest job's site count;
   the second serves admissions and read-backs while a chunk runs), the rest
   is the job heap.  No other device memory is used; the batch creates one
   side stream of its own and an 8-byte pinned host word. */
typedef struct smcx_batch smcx_batch;

/* Bytes of the arena's control area; 0 for max_jobs == 0. */
size_t smcx_batch_control_bytes(uint32_t max_jobs, size_t transfer_bytes);

/* Heap bytes one job of this descriptor occupies (0 if invalid). */
size_t smcx_batch_job_bytes(const smcx_lattice_desc* desc);

/* Binds the arena and the stream (a cudaStream_t; with a non-NULL stream
   chunks are captured into CUDA graphs).  ENOMEM: arena smaller than the
   control area. */
smcx_status smcx_batch_create(uint32_t max_jobs, void* d_arena, size_t arena_bytes,
                              size_t transfer_bytes, void* cuda_stream, smcx_batch** out);

/* Admits a job: occupancy h_init (canonical, N bytes), EPI [n_shells][K][K]
   (q units, symmetric), temperature T (kelvin, constant), n_sweeps to run.
   The job starts at sweep counter 0 and joins the next chunk
   (smcx_batch_run or smcx_batch_launch).  While a launched chunk runs, the
   upload and the job's initial energy go through the batch's side stream
   and a second transfer buffer, overlapping the chunk on the device (the
   call still returns only when the job is admitted).  *job_id receives its
   id (a slot index, reused after smcx_batch_remove).  EBUDGET: no free slot
   or no room left in the arena.  EINVAL: invalid or unsupported job. */
smcx_status smcx_batch_add(smcx_batch* b, const smcx_lattice_desc* desc, const uint8_t* h_init,
                           uint32_t n_shells, const int64_t* v_q, double T, uint32_t n_sweeps,
                           uint32_t* job_id);

/* Runs up to chunk_sweeps sweeps of every active job (fewer for jobs that
   finish inside the chunk) and synchronises.  *n_finished (may be NULL)
   receives the number of jobs that completed in this chunk.  While the
   batch is untuned, the first sweeps run as short timed sub-chunks, one per
   tuning candidate (results are unaffected).  ETIMEOUT: a device-side wait
   gave up (the batch then stays in an error state). */
smcx_status smcx_batch_run(smcx_batch* b, uint32_t chunk_sweeps, uint32_t* n_finished);

/* The same chunk split in two, so that host work overlaps the device:
   smcx_batch_launch enqueues up to chunk_sweeps sweeps of every active job
   on the batch's stream and returns at once (first completing a chunk still
   in flight); smcx_batch_wait completes the chunk in flight and *n_finished
   (may be NULL) receives the number of jobs finished since the last report.
   Results are those of smcx_batch_run.  Between the two calls,
   smcx_batch_add admits jobs for the next chunk and smcx_batch_result /
   smcx_batch_remove serve jobs that finished earlier, through the side
   stream; smcx_batch_poll reports jobs finished by completed chunks only.
   Calls that need the running jobs (their results, exchange, queue
   statistics, smcx_batch_run) complete the chunk first.  While the batch is
   still tuning, smcx_batch_launch runs its chunk to completion (the tuning
   times it).  ETIMEOUT as for smcx_batch_run. */
smcx_status smcx_batch_launch(smcx_batch* b, uint32_t chunk_sweeps);
smcx_status smcx_batch_wait(smcx_batch* b, uint32_t* n_finished);

/* Tuning of the batched sweep (never changes results):
     SMCX_BATCH_OPT_TILE       work-item shape index (see smcx_batch_tile_shape)
     SMCX_BATCH_OPT_SCHEDULE   0 = persistent plan (one cooperative launch
                               per chunk, per-job phase counters), 1 = one
                               launch per colour phase for all jobs
     SMCX_BATCH_OPT_OCCUPANCY  register budget index: 0, 1 = 3, 4 resident
                               blocks of 128 threads per SM
   Value -1 (the default) = chosen online.  Setting any restarts the online
   tuning. */
#define SMCX_BATCH_OPT_TILE 1u
#define SMCX_BATCH_OPT_OCCUPANCY 2u
#define SMCX_BATCH_OPT_SCHEDULE 3u
/* Testing aid for failure detection (value 1 arms it): the next run with the
   persistent schedule tells the kernel that the first active job has
   one work item per phase more than it has, so the waits for that job's
   earlier phases give up after their limit (about 2 s); the run returns
   ETIMEOUT and the batch stays in an error state.  Nothing faults or hangs. */
#define SMCX_BATCH_OPT_TEST_WAIT_TIMEOUT 4u
smcx_status smcx_batch_set_option(smcx_batch* b, uint32_t key, int64_t value);

/* Current choice: *tile, *schedule and *occupancy (-1 while tuning), *tuned
   = 1 once the online tuning has finished.  Any pointer may be NULL. */
smcx_status smcx_batch_tuning(smcx_batch* b, int32_t* tile, int32_t* schedule, int32_t* occupancy,
                              uint32_t* tuned);

/* Replica exchange (parallel tempering, Sec. 2.2, Eqs. 6-7) between jobs
   that simulate the same system (same descriptor, shells and EPI) at
   different temperatures.  ladder[0..n) (in/out) = job ids, ladder[k] being
   the job at the k-th temperature of the ladder.  Round `round` attempts the
   neighbour pairs (k, k+1) for k = round mod 2, round mod 2 + 2, ...:
   Delta = (beta_k - beta_{k+1}) (E_k - E_{k+1}), beta = 1/(k_B T) (k_B =
   8.617333262e-5 eV/K), E the jobs' exact running energies (q units; the
   difference is formed in integers and scaled by 2^-32 to eV); accepted iff
   Delta >= 0 or u < exp(Delta), u in [0, 1) from the 53 high bits of words
   0 and 1 of Philox4x32-10(counter = (k, round, 0, 3), key = seed).  An
   accepted pair exchanges the two jobs' temperatures and their ladder
   entries (so ladder[k] is again the job at the k-th temperature).
   *n_accepted (may be NULL) = accepted pairs.  Call between runs; it
   synchronises.  EINVAL: fewer than 2 jobs, unknown or repeated ids, jobs
   of different systems, a temperature that is 0 or infinite. */
smcx_status smcx_batch_exchange(smcx_batch* b, uint32_t* ladder, uint32_t n, uint64_t seed,
                                uint32_t round, uint32_t* n_accepted);

/* Current temperature of a job (changes through smcx_batch_exchange). */
smcx_status smcx_batch_temperature(smcx_batch* b, uint32_t job_id, double* T);

/* Persistent-schedule statistics since the batch was created: out[0] =
   item ranges that had to wait for the previous colour phase of their job,
   out[1] = polls of those waits, out[2] = nanoseconds they waited (summed
   over warps).  Synchronises. */
smcx_status smcx_batch_queue_stats(smcx_batch* b, uint64_t* out);

/* Active link cells (x, y, z) of work-item shape i (product 32): shape 0
   is 32 consecutive cells of a colour in x-fastest order (rows wrap, so
   (32, 1, 1) only when a row has >= 32), shapes 1..3 are boxes.  EINVAL for
   i >= 4. */
smcx_status smcx_batch_tile_shape(uint32_t i, uint32_t* cells_xyz);

/* Pops up to cap ids of finished jobs (completion order) into ids; *n gets
   the count. */
smcx_status smcx_batch_poll(smcx_batch* b, uint32_t* ids, uint32_t cap, uint32_t* n);

/* Result of a job (finished or not): occupancy (canonical, N bytes; h_occ
   may be NULL), cumulative trial statistics, running energy (q units) and
   sweeps done.  Synchronises. */
smcx_status smcx_batch_result(smcx_batch* b, uint32_t job_id, uint8_t* h_occ,
                              smcx_sweep_stats* totals, int64_t* e_run, uint32_t* sweeps_done);

/* Releases a job's slot and heap space. */
smcx_status smcx_batch_remove(smcx_batch* b, uint32_t job_id);

/* Occupancy of the batch: running jobs, free slots, free heap bytes and the
   largest free block. */
smcx_status smcx_batch_info(smcx_batch* b, uint32_t* active, uint32_t* free_slots,
                            size_t* free_bytes, size_t* largest_free);

smcx_status smcx_batch_destroy(smcx_batch* b);

/* ---- pair counts without allocation ---------------------------------------
   (No counterpart in the paper: an interface for callers that cannot
   allocate device memory where they need the counts -- code running inside
   another framework's memory-pool callbacks or allocator hooks, where a
   nested allocation would recurse or deadlock; processes whose device memory
   is wholly reserved by their host framework; deployments that forbid
   allocation after start-up.)

   Computes the same directed shell pair counts N_m[p'][p] as
   smcx_warren_cowley_sro, from a caller's device occupancy in the canonical
   layout (d_canon, N bytes), into the caller's device array d_counts
   ([n_shells][K][K] uint64), enqueued on cuda_stream (a cudaStream_t,
   NULL = legacy default stream); the call does not synchronise.  It needs
   no handle and no workspace and never allocates: its accumulators live in
   a static device array of the library holding SMCX_NOALLOC_MAX_SHELLS x
   SMCX_NOALLOC_MAX_SPECIES^2 counters (8 KiB), which every GPU that loads
   the library keeps until the process exits.  Every call looks up that
   array's device address for the current device and context
   (cudaGetSymbolAddress, a host-side query; a kept address could outlive a
   cudaDeviceReset).  The first call on a device also loads the library's
   module there, so make it before any stream capture.  All calls on a device
   share the array, which is cleared at the start of each call and keeps the
   last call's counts afterwards: calls whose work overlaps on the GPU (other
   streams, other threads) race and must be serialised by the caller.  Pairs
   involving a site whose id is >= n_species are not counted.
   EINVAL: kind not BCC/FCC, n_species > 16, n_shells outside 1..4, a size
   of 0, 2^32 or more sites, or a null pointer.  ECUDA: symbol lookup or
   launch failed. */
#define SMCX_NOALLOC_MAX_SHELLS 4
#define SMCX_NOALLOC_MAX_SPECIES 16
smcx_status smcx_pair_counts_noalloc(uint32_t kind, const uint32_t* n, uint32_t n_species,
                                     uint32_t n_shells, const uint8_t* d_canon, uint64_t* d_counts,
                                     void* cuda_stream);

/* Shell table used by the library: writes up to cap vectors (dx,dy,dz in
   half units) of shells 1..n_shells, sorted by distance then
   lexicographically, and z[m]; returns the number of vectors, 0 on error. */
uint32_t smcx_shell_table(uint32_t kind, uint32_t n_shells, int32_t* disp, uint32_t cap,
                          uint32_t* z);

/* Philox4x32-10 of the library (for cross-checks): out[4] for the counter
   ctr[4] and key[2]; runs on the host. */
void smcx_philox4x32_10(const uint32_t* ctr, const uint32_t* key, uint32_t* out);

/* Same generator evaluated by the library's device code: for i < n, writes
   Philox4x32-10 of counter (c0 + i, c1, c2, c3) under key to d_out[4*i..].
   d_out: device, 4*n uint32.  Synchronises the given stream. */
smcx_status smcx_philox_device(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint64_t key,
                               uint32_t n, uint32_t* d_out, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* SMCX_H */
