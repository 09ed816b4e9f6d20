/*
 * ml.h -- C ABI of the B300 multilevel Monte Carlo library (libml.so) for
 * d = 3+1 compact U(1) Wilson-action lattice gauge theory.
 *
 * The library runs the Luescher-Weisz multilevel algorithm as used by Amado,
 * Cardoso & Bicudo, arXiv:1309.3859 (Section II.C and Algorithm 1):
 * checkerboard heatbath + overrelaxation sweeps with the spatial links of slab
 * boundaries frozen, per-slab averages of two-link Polyakov factors with and
 * without a plaquette field insertion, and cross-slab products that give the
 * Polyakov-loop correlator P(r) and the flux-tube field profile.
 *
 * Conventions used by every entry point:
 *   site index  i = x + L*(y + L*(z + L*t)), periodic in all four directions;
 *   direction   0 = t (the paper's U_0), 1 = x, 2 = y, 3 = z;
 *   angles      U_mu(i) = exp(i theta_mu(i)); host angle buffers hold
 *               theta[mu * V + i] in double precision (V = L^3 Nt);
 *   components  c = 0..5 are Ex, Ey, Ez, Bx, By, Bz = the plaquettes
 *               P_01, P_02, P_03, P_23, P_31, P_12 (Section II.B);
 *   charges     static charge at x, anti-charge at x + r xhat.
 *
 * Errors: every function returns an ml_status (0 = ML_OK, negative = error).
 * No function throws across the ABI.  After ML_ETIMEOUT or ML_EREJECT the
 * handle stays valid for inspection and ml_destroy.
 *
 * Streams: all device work of a handle is enqueued on the stream given to
 * ml_create.  Functions documented as blocking synchronise that stream.
 */
#ifndef ML_H
#define ML_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  ML_OK = 0,
  ML_EINVAL = -1,   /* invalid argument or parameter set                      */
  ML_ENOMEM = -2,   /* the allocator returned NULL                            */
  ML_ECUDA = -3,    /* a CUDA runtime call failed                             */
  ML_ETIMEOUT = -4, /* a bounded device wait gave up                          */
  ML_EREJECT = -5,  /* the von Mises rejection loop reached its trial cap     */
  ML_EBUSY = -6,    /* resource in use (e.g. server at capacity)              */
  ML_ESTATE = -7    /* call not allowed in the handle's state                 */
} ml_status;

typedef enum {
  ML_FP64 = 0, /* link angles and update arithmetic in double precision       */
  ML_FP32 = 1  /* link angles, update arithmetic and the per-sub-update
                  records (slab phase sums, plaquette slab sums) in single
                  precision; each fold adds the single-precision sum of a
                  batch of up to 16 sub-update terms to double-precision slab
                  sums; slab averages, level combination, cross-slab products,
                  reductions over sites and final ratios in double precision
                  (pair_sums = 1 keeps the slab sums as float pairs instead)  */
} ml_precision;

/* Transverse offset (dy, dz) of a field probe from the mid-point of the
 * charges (the paper's mediator plane, Section III.B). */
typedef struct {
  int dy, dz;
} ml_offset;

/* Update of the first sweep of every compound sweep. */
typedef enum {
  ML_UPDATE_HEATBATH = 0,  /* exact draw of the link's conditional law (Best & Fisher sampler) */
  ML_UPDATE_METROPOLIS = 1 /* Section II's Metropolis: metro_hits hits per link, proposal
                              theta + w (2 u1 - 1) with w = metro_width, accepted when
                              u2 < exp(beta k [cos(theta' + alpha) - cos(theta + alpha)]);
                              (u1, u2) are those of heatbath trial h of the same stream */
} ml_update;

/* Run parameters.  Validation (ML_EINVAL): L and Nt even and >= 2, L^3 Nt <=
 * 2^30, Nt <= 2^20; slab >= 1
 * dividing Nt; n_sub >= 1; outer_slab = 0, or a multiple of slab that divides
 * Nt and differs from slab, with n_sub_outer >= 1; 1 <= r, rf <= L-1;
 * |dy|, |dz| <= L-1; beta >= 0; k_between >= 0; n_or >= 0; comp_mask < 64;
 * at least one r; update an ml_update, and for Metropolis 1 <= metro_hits <= 64
 * and 0 < metro_width <= pi; multihit 0 or 1, with multihit beta <= 100;
 * replay 0 or 1, with replay outer_slab = 0; pair_sums 0, or 1 with prec =
 * ML_FP32.  The lists are copied by ml_create. */
typedef struct {
  int L, Nt;            /* spatial and temporal extent                         */
  double beta;          /* inverse coupling 1/g^2 of the Wilson action         */
  uint64_t seed;        /* key of the Philox stream                            */
  int prec;             /* ml_precision                                        */
  int n_or;             /* overrelaxation sweeps per heatbath sweep (paper: 3) */
  int slab;             /* inner slab thickness d (paper: 2)                   */
  int n_sub;            /* inner sub-updates n2 per (outer) iteration          */
  int outer_slab;       /* 0: one level; else outer thickness (paper: 4)       */
  int n_sub_outer;      /* outer sub-updates n4                                */
  int k_between;        /* full compound sweeps before each measurement, k0    */
  int nr;               /* number of P(r) separations                          */
  const int *r;         /* P(r) separations along x                            */
  int nrf;              /* number of field-profile separations                 */
  const int *rf;        /* separations of the field profile                    */
  int nprobe;           /* number of probe offsets                             */
  const ml_offset *probe; /* probe offsets on the mediator plane               */
  uint32_t comp_mask;   /* bit c selects field component c                     */
  int update;           /* ml_update of the first sweep of a compound sweep    */
  int metro_hits;       /* Metropolis hits per link visit                      */
  double metro_width;   /* Metropolis proposal half-width (radians)            */
  int multihit;         /* 1: analytic multihit of the temporal links in P(r)
                           at 2 <= r <= L-2 (Section II.C): each link of the
                           two lines in a slab is replaced by its conditional
                           mean e^{-i alpha} I1(beta k) / I0(beta k), k e^{i alpha}
                           its staple sum; the field profile keeps the plain
                           links                                               */
  int replay;           /* 1: field insertions by replay (one level only): the
                           inner loop runs twice from the same configuration
                           and sweep numbers, first forming the slab averages
                           [T], then adding every sub-update's T O times the
                           other slabs' [T] straight into the products, so no
                           per-site [TO] sums are kept (same estimator, the
                           field-insertion memory for twice the slab sweeps) */
  int pair_sums;        /* ML_FP32 only.  0 (default): slab sums in double
                           precision.  1: each slab sum kept as an unevaluated
                           sum hi + lo of two binary32 numbers (about 47
                           significant bits; error-free additions on the
                           single-precision pipe, which this GPU runs far
                           faster than its double-precision one); averages,
                           products and reductions stay double precision      */
} ml_params;

/* Device-memory allocator supplied by the caller (the Python binding passes
 * PyTorch's caching allocator).  alloc returns device memory of at least
 * `bytes` bytes aligned to 256 bytes, or NULL; free releases it. */
typedef struct {
  void *(*alloc)(size_t bytes, void *ctx);
  void (*free)(void *ptr, void *ctx);
  void *ctx;
} ml_allocator;

typedef struct ml_lattice ml_lattice;

/* ------------------------------------------------------------------------ */
/* Lattice lifecycle                                                          */
/* ------------------------------------------------------------------------ */

/* Validates *p, allocates the lattice through *alloc (NULL: cudaMalloc) on
 * the current device, and enqueues the hot start theta = -pi + 2 pi u on
 * `cuda_stream` (a cudaStream_t; NULL = legacy default stream).  u is the
 * 52-bit uniform of Philox block (i, mu, 0, 0) keyed by the seed.  Sweep
 * numbering starts at 1 with the first heatbath sweep.  Ownership of the
 * handle passes to the caller; release it with ml_destroy. */
int ml_create(const ml_params *p, const ml_allocator *alloc, void *cuda_stream, ml_lattice **out);

/* Synchronises the handle's stream and frees everything it owns. */
int ml_destroy(ml_lattice *h);

/* n_sweeps compound sweeps (one heatbath sweep + n_or overrelaxation sweeps,
 * Section II) with no frozen links: thermalisation (Section II, Algorithm 1's
 * k0 loop).  Asynchronous; errors surface at the next blocking call. */
int ml_thermalize(ml_lattice *h, int n_sweeps);

/* n_meas multilevel measurements (Algorithm 1).  Each one runs k_between full
 * compound sweeps, then the slab sub-updates with frozen boundary spatial
 * links (one level: n_sub sub-updates of thickness `slab`; two levels:
 * n_sub_outer iterations of one outer sweep plus n_sub inner sub-updates),
 * accumulating the slab averages of T^(d) and TO^(d) (Section II.C), then the
 * cross-slab products.  Blocks until the records are in out_host.
 * out_host receives n_meas records of ml_record_len doubles (layout below);
 * out_len is its capacity in doubles. */
int ml_measure(ml_lattice *h, int n_meas, double *out_host, size_t out_len);

/* Same as ml_measure but leaves the records in device memory out_dev
 * (n_meas * record_len doubles) and does not synchronise. */
int ml_measure_device(ml_lattice *h, int n_meas, double *out_dev, size_t out_len);

/* Doubles of one measurement record for parameter set *p:
 *   P      [nr][2]               (Re, Im) (1/Ns) sum_x prod_s [T]_s(x, r)
 *   Pf     [nrf][2]              the same at the field separations
 *   W      [nrf][nprobe][6][2][2] for component c and insertion k (0: Re P_c,
 *                                1: Im P_c), (Re, Im) of (1/(Ns Nt)) sum_x
 *                                sum_s [TO]_s prod_{s' != s} [T]_{s'}
 *   vac    [6][2]                mean Re P_c, Im P_c over sites and the
 *                                sub-update configurations
 *   naive  [nr][2]               (1/Ns) sum_x P(x)^* P(x + r) on the first
 *                                configuration of the measurement
 *   plaq   [1]                   mean plaquette of that configuration
 * Unselected components are zero.  Ns = L^3. */
int ml_record_len(const ml_params *p, size_t *len);

/* Connected field profile from n_meas records already in device memory
 * (Section II.C, electromagnetic-field equations): with means over measurements,
 *   F   = sqrt(beta) ( <Re W_{c,1}> / <Re Pf> - <vac_{c,1}> )
 *   F^2 = -2 beta   ( <Re W_{c,0}> / <Re Pf> - <vac_{c,0}> )
 * written as out_dev[nrf][nprobe][6][2] (F, F^2), computed in double
 * precision on the device.  Asynchronous on the handle's stream. */
int ml_connected_device(ml_lattice *h, const double *records_dev, int n_meas, double *out_dev, size_t out_len);

/* ------------------------------------------------------------------------ */
/* Configuration access and single steps (checkpointing, tests)              */
/* ------------------------------------------------------------------------ */

/* Copies the angles to / from host memory theta[4 * V] (double, canonical
 * layout above).  Blocking.  ml_set_angles wraps values into [-pi, pi). */
int ml_get_angles(ml_lattice *h, double *theta_host, size_t n);
int ml_set_angles(ml_lattice *h, const double *theta_host, size_t n);

/* Number of heatbath sweeps done so far (the Philox sweep counter); setting
 * it with the saved angles resumes a run bit-exactly. */
int ml_get_sweep(ml_lattice *h, uint64_t *n);
int ml_set_sweep(ml_lattice *h, uint64_t n);

/* One pass over the links U_mu(x) of parity `parity` (0 even, 1 odd) that
 * are not frozen (slab_d > 0 freezes spatial links on t = 0 mod slab_d):
 * kind 0 = the handle's update (heatbath or Metropolis) with sweep number n,
 * kind 1 = overrelaxation, kind 2 = Metropolis (handles created with
 * ML_UPDATE_METROPOLIS only, else ML_EINVAL).  Asynchronous.  Does not change
 * the sweep counter. */
int ml_update_pass(ml_lattice *h, int mu, int parity, int slab_d, uint64_t n, int kind);

/* n compound sweeps with slab mask slab_d (0 = none). Asynchronous. */
int ml_compound_sweeps(ml_lattice *h, int n, int slab_d);

/* Record (layout of ml_record_len) of the current configuration alone, as a
 * measurement with one sub-update and no sweep.  Blocking. */
int ml_observe(ml_lattice *h, double *out_host, size_t out_len);

/* Waits for the handle's stream and reports deferred device errors. */
int ml_sync(ml_lattice *h);

/* ------------------------------------------------------------------------ */
/* Time-slab partition of one lattice over several processes                 */
/* ------------------------------------------------------------------------ */

/* Section II.C: with the spatial links of the slab boundaries frozen, the
 * slabs' sub-updates are independent of one another.  A lattice can
 * therefore be split by time slices over R processes (one GPU each), every
 * process holding the whole lattice but moving only the links of its own
 * slices [t_lo, t_hi).  One measurement then runs as:
 *   1. k0 full compound sweeps, pass by pass (ml_update_pass), from
 *      boundary slices refreshed in every direction and parity (the previous
 *      measurement's sub-updates moved the neighbours' boundary links), each
 *      pass followed by the exchange of the moved links on the two boundary
 *      slices with the neighbouring processes (ML_PART_LINKS);
 *   2. the owned slices of every process gathered into every copy, so each
 *      copy is the whole configuration (ML_PART_LINKS);
 *   3. ml_measure_inner: naive correlator and plaquette of that
 *      configuration, the slab sub-updates, records and folds of the owned
 *      slabs (no exchange at all);
 *   4. the top-level [T] slab sums (ML_PART_SLAB_SUMS) of every process
 *      gathered into every copy (each process's products multiply by the
 *      other slabs' averages), the vacuum block sums (ML_PART_VACUUM) into
 *      the copy of the process with the last slabs;
 *   5. ml_measure_products in process order: each adds its slabs' field
 *      insertions to the per-site sums it receives and passes them on
 *      (ML_PART_W_SUMS bytes); the last reduces them into the record.
 * The records are bit-identical to those of one process running ml_measure
 * (the same kernels add the same terms in the same order).  The exchanges
 * are the caller's (the Python binding's partition module uses
 * torch.distributed).  While a range other than the whole lattice is set,
 * ml_thermalize and ml_measure return ML_ESTATE. */

/* Own the time slices [t_lo, t_hi): t_lo and t_hi multiples of the top-level
 * slab thickness (outer_slab for two levels, else slab), 0 <= t_lo < t_hi <=
 * Nt; (0, Nt) restores the whole lattice.  Handles with replay: ML_EINVAL.
 * Blocking (re-plans the sweeps and re-captures the graphs). */
int ml_set_time_range(ml_lattice *h, int t_lo, int t_hi);

typedef enum {
  ML_PART_LINKS = 0,     /* one time slice of the links of one direction and parity:
                            L^3 / 2 angles in the lattice's precision           */
  ML_PART_SLAB_SUMS = 1, /* one top-level slab's [T] sums: nR L^3 complex values of
                            16 bytes (nR: the distinct separations of r and rf)  */
  ML_PART_VACUUM = 2,    /* one inner slab's vacuum block sums (doubles)          */
  ML_PART_W_SUMS = 3     /* the per-site field-insertion sums passed between
                            processes: nrf nprobe nc 2 L^3 complex values of 16 bytes
                            (nc: selected components); ml_part_size only        */
} ml_part_block;

/* Bytes of one unit of block `what` (a slice, a slab; for ML_PART_W_SUMS the
 * whole array). */
int ml_part_size(ml_lattice *h, int what, size_t *bytes);

/* Copies units [begin, begin + count) of block `what` (for ML_PART_LINKS
 * direction mu and parity `parity`, slices begin.. of that array) between the
 * lattice and the device buffer buf_dev (to_lattice = 1: buffer -> lattice),
 * on the handle's stream after its accumulation work.  Asynchronous. */
int ml_part_copy(ml_lattice *h, int what, int mu, int parity, int begin, int count, void *buf_dev, int to_lattice);

/* Step 3 above; rec_dev (rec_len >= ml_record_len doubles of device memory)
 * receives the naive and plaquette blocks.  Asynchronous. */
int ml_measure_inner(ml_lattice *h, double *rec_dev, size_t rec_len);

/* Step 5 above: w_in_dev (NULL: zero; ML_PART_W_SUMS bytes) are the sums of
 * the preceding processes.  With w_out_dev the sums after this process's
 * slabs go there and rec_dev is not touched; with w_out_dev = NULL the
 * record's P, Pf, W and vacuum blocks are completed in rec_dev.  ML_ESTATE
 * without a preceding ml_measure_inner.  Asynchronous. */
int ml_measure_products(ml_lattice *h, const void *w_in_dev, void *w_out_dev, double *rec_dev, size_t rec_len);

/* ------------------------------------------------------------------------ */
/* Utilities                                                                  */
/* ------------------------------------------------------------------------ */

/* Philox4x32-10 (Salmon et al., SC'11) evaluated on the device for n
 * counters ctr[4n] and keys key[2n] (host arrays); out[4n] on the host.
 * Blocking.  Used to check the device generator bit for bit. */
int ml_philox(const uint32_t *ctr, const uint32_t *key, size_t n, uint32_t *out);

/* Self-check of the single-precision link update's own rounding (no
 * counterpart in the paper: an implementation detail).  The FP32 update
 * rounds its range reductions and its wrap to [-pi, pi) by adding and
 * subtracting 1.5 2^23 on the FP32 pipe instead of rintf / floorf, and builds
 * its uniforms (k + 1/2) 2^-p in the mantissa instead of converting k.  This
 * counts, on the device, the values where they differ from the conversions:
 * mismatches[0] rint and mismatches[1] floor over every float of magnitude
 * below 2^22, mismatches[2] every 23-bit uniform, mismatches[3] 2^24 52-bit
 * uniforms spread over the range (a zero result of either sign counts as
 * equal to the other).  All four are 0 on a correct build.
 * mismatches: host array of 4.  Blocking; allocates 32 bytes on the current
 * device.  ML_ECUDA on a CUDA error. */
int ml_check_rounding(unsigned long long *mismatches);

/* Kernel classes of ml_kernel_timing. */
typedef enum {
  ML_K_HEATBATH = 0,   /* one heatbath pass kernel (mu = 1, even sites, slab mask) */
  ML_K_OVERRELAX = 1,  /* one overrelaxation pass kernel (same links)             */
  ML_K_RECORD = 2,     /* record of one sub-update: slab phase and plaquette sums */
  ML_K_ACCUMULATE = 3, /* fold of a full batch of records into the slab sums      */
  ML_K_PRODUCTS = 4,   /* cross-slab products and their reduction over sites      */
  ML_K_SWEEP = 5,      /* one compound slab sweep (the handle's implementation)   */
  ML_K_SUBUPDATE = 6,  /* one slab sub-update as measurements run it: compound
                          sweep and record (fused in the persistent and
                          resident kernels; the resident kernel runs a ring
                          buffer of sub-updates per launch, and the time is
                          that launch's divided by its sub-updates)           */
  ML_K_FULLSWEEP = 7   /* one compound sweep without frozen links, as between
                          measurements and in ml_thermalize                     */
} ml_kernel_class;

/* Average device time in milliseconds of `reps` back-to-back launches of one
 * kernel class, bracketed by CUDA events on the handle's stream, in the
 * launch configuration ml_measure uses.  Update passes run on a scratch copy
 * of the angles, so the Markov chain is unchanged; the slab accumulators are
 * left undefined (every measurement clears them first).  Blocking. */
int ml_kernel_timing(ml_lattice *h, int kernel, int reps, double *avg_ms);

/* Launch timeline of the measurement schedule (Algorithm 1 as ml_measure and
 * ml_measure_device enqueue it): with a capacity set, CUDA events are
 * recorded around the full sweeps between measurements, every sub-update
 * group (one cluster-resident launch of a ring buffer of sub-updates, or a
 * ring buffer's worth of per-pass or persistent sub-update graphs) and the
 * loop's last group, on the main stream, and around every fold of a ring
 * buffer and the products, on the accumulation stream, until the capacity is
 * used up.  The events only time: the schedule and the results are
 * unchanged.  ml_timeline_enable(h, 0) turns it off; a new capacity discards
 * earlier marks. */
typedef enum {
  ML_TL_FULL_BEGIN = 0, /* k0 full sweeps of a measurement (main stream)   */
  ML_TL_FULL_END = 1,
  ML_TL_SUB_BEGIN = 2,  /* a group of slab sub-updates (main stream)        */
  ML_TL_SUB_END = 3,
  ML_TL_FOLD_BEGIN = 4, /* the fold of a ring buffer (accumulation stream)  */
  ML_TL_FOLD_END = 5,
  ML_TL_PROD_BEGIN = 6, /* the products of a measurement, with the last
                           buffer's field insertions (accumulation stream)  */
  ML_TL_PROD_END = 7
} ml_timeline_tag;
int ml_timeline_enable(ml_lattice *h, int capacity);
/* Waits for the handle's streams, then writes up to cap marks in recording
 * order: tags[i] (ml_timeline_tag) and ms[i], the device time of mark i
 * after the first mark; *n = the number written.  The marks are then
 * discarded (the capacity stays). */
int ml_timeline_read(ml_lattice *h, int *tags, float *ms, int cap, int *n);

/* Where the cluster-resident sub-updates spend their time: one launch as a
 * measurement runs it (a ring buffer of sub-updates with their records, on
 * the timing copy of the angles, so the chain is unchanged) in a variant in
 * which thread 0 of every CTA reads the SM clock around its phases, with a
 * block barrier between a pass's own link updates and its exchange.  out
 * (ML_RESIDENT_PROFILE_LEN doubles, SM clock cycles averaged over the CTAs):
 *   [0..3]  own link updates per pass, pass classes heatbath mu = 0,
 *           heatbath mu > 0, overrelaxation mu = 0, overrelaxation mu > 0
 *   [4..7]  exchange per pass (waiting for the neighbours' mirror stores and
 *           tokens of the pass, and the block barrier after it), same classes
 *   [8]     record of one sub-update (phase and plaquette sums, with its
 *           cluster barriers)
 *   [9]     launch set-up (box load, mirror lists, cluster barriers)
 *   [10]    write-back of the links
 *   [11]    the whole launch
 *   [12]    sub-updates in the launch
 *   [13]    CTAs
 * ML_EINVAL when the handle's sub-updates are not cluster-resident.
 * Blocking. */
#define ML_RESIDENT_PROFILE_LEN 14
int ml_resident_profile(ml_lattice *h, double *out, int n);

/* Implementations of the compound sweep.  ml_create times the available
 * ones on the handle's lattices and keeps the fastest; results are
 * bit-identical. */
typedef enum {
  ML_SWEEP_PERSISTENT = 0, /* one cooperative persistent kernel, grid barrier
                              (bounded spin) between passes                   */
  ML_SWEEP_PASSES = 1,     /* one kernel per (direction, parity) pass, replayed
                              from a CUDA graph                               */
  ML_SWEEP_RESIDENT = 2    /* slab sub-updates: one thread-block cluster per
                              time slab keeps the slab's links in distributed
                              shared memory, hardware cluster barrier between
                              passes; available when a slab fits the cluster's
                              shared memory (else ML_EINVAL when forced).
                              Sweeps without frozen links run as the faster of
                              the other two.                                  */
} ml_sweep_impl;

/* Query or force the compound-sweep implementation (forcing re-captures the
 * handle's graphs; blocking). */
int ml_sweep_mode(ml_lattice *h, int *mode);
int ml_set_sweep_mode(ml_lattice *h, int mode);

/* Implementation of the field-insertion fold (Section II.C's [TO] sums). */
typedef enum {
  ML_FOLD_SITE = 0, /* one thread per site reads each probe's recorded plaquette sums from global memory */
  ML_FOLD_TILE = 1  /* a block stages the recorded plaquette sums its probes reach in shared memory once
                       per component; available when every lattice has L <= 256 and a tile of at most
                       96 KB (else ML_EINVAL when forced) */
} ml_fold_impl;
/* Query or force the fold implementation; ml_create picks the faster of the
 * two on the handle's table.  Both give bit-identical sums. */
int ml_fold_mode(ml_lattice *h, int *mode);
int ml_set_fold_mode(ml_lattice *h, int mode);

/* Number of sub-update records the handle folds into its slab sums per
 * accumulation pass (chosen at ml_create from the record size, at most 16). */
int ml_batch_slots(ml_lattice *h, int *n);

/* ------------------------------------------------------------------------ */
/* Batches: many independent lattices advanced together                      */
/* ------------------------------------------------------------------------ */

/* A batch holds n independent lattices (different L, Nt, beta, seed,
 * separations, probes and components) that share one schedule: precision,
 * n_or, slab, outer_slab, n_sub, n_sub_outer, k_between and replay must be
 * equal (else ML_EINVAL).  Every sweep, record and fold of the batch is one kernel
 * launch over all its lattices (the multi-lattice kernels a single lattice
 * also runs), so each lattice's results are identical to those of the same
 * parameters run alone with ml_create.  Memory and stream as for ml_create. */
typedef struct ml_batch ml_batch;
int ml_batch_create(const ml_params *ps, int n, const ml_allocator *alloc, void *cuda_stream, ml_batch **out);
int ml_batch_destroy(ml_batch *b);
int ml_batch_size(ml_batch *b, int *n);
/* n_sweeps full compound sweeps of every lattice.  Asynchronous. */
int ml_batch_thermalize(ml_batch *b, int n_sweeps);
/* n_meas measurements of every lattice (Algorithm 1).  Output layout:
 * lattice-major, [lattice][measurement][record of that lattice], total
 * length from ml_batch_result_len, lattice offsets from
 * ml_batch_record_offset.  ml_batch_measure blocks; the _device variant
 * writes device memory asynchronously. */
int ml_batch_result_len(ml_batch *b, int n_meas, size_t *len);
int ml_batch_record_offset(ml_batch *b, int lattice, int n_meas, size_t *offset);
int ml_batch_measure(ml_batch *b, int n_meas, double *out_host, size_t out_len);
int ml_batch_measure_device(ml_batch *b, int n_meas, double *out_dev, size_t out_len);
int ml_batch_get_angles(ml_batch *b, int lattice, double *theta_host, size_t n);
int ml_batch_sync(ml_batch *b);
int ml_batch_sweep_mode(ml_batch *b, int *mode);
int ml_batch_set_sweep_mode(ml_batch *b, int mode);

/* ------------------------------------------------------------------------ */
/* Serving: measurement requests with continuous batching                     */
/* ------------------------------------------------------------------------ */

/* A server owns one device allocation of budget_bytes (the HBM budget) and
 * `lanes` size lanes, each with its own stream and worker thread; a request
 * goes to the lane of its lattice volume V = L^3 Nt (with three lanes: V below
 * 2^16 sites, below 2^18, and the rest), so small requests do not wait on the
 * ticks of large ones and the lanes' launches overlap on the GPU.  Requests
 * (one lattice each: create, n_therm thermalisation sweeps, n_meas
 * measurements) are admitted first-in first-out within a lane whenever their
 * memory fits the budget and fewer than max_active (0: 1024) are running in
 * all lanes.  The admitted lattices of a lane advance together: each worker
 * tick is one launch in which every lattice advances by its share of compound
 * sweeps (the lane's largest volume over its own, at most 2, within its
 * phase; inner sub-updates recorded into consecutive ring slots), one fold
 * launch over the lattices that need it, and the per-lattice steps of
 * Algorithm 1.  Requests that arrive while others run join at the next tick;
 * finished ones leave and free their memory.  Each request's records are
 * identical to the same parameters run with ml_create.  All requests of a
 * server share prec and n_or. */
typedef struct {
  int prec;            /* ml_precision of every request                      */
  int n_or;            /* overrelaxation sweeps per heatbath sweep           */
  size_t budget_bytes; /* device memory for all resident requests (>= 1 MiB) */
  int max_active;      /* bound on simultaneously resident requests (0: 1024) */
  int lanes;           /* size lanes, 1..8 (0: 3)                            */
} ml_server_config;

typedef struct {
  int queued, active;
  uint64_t completed, failed, ticks;
  size_t budget_bytes, used_bytes;
} ml_server_info;

typedef struct ml_server ml_server;
/* Allocates the budget (cudaMalloc, current device) and starts the worker. */
int ml_server_create(const ml_server_config *cfg, ml_server **out);
/* Queues a request (parameters are copied); *job identifies it.  ML_EINVAL
 * for invalid parameters, a precision / n_or different from the server's, or
 * replay (the server folds every record as it comes).
 * A request that cannot fit the budget even alone completes with ML_ENOMEM. */
int ml_submit(ml_server *s, const ml_params *p, int n_therm, int n_meas, uint64_t *job);
/* Non-blocking: *done = 1 once the request has finished.  When done and
 * out_host is not NULL, copies its n_meas records (ml_record_len layout).
 * Returns the request's status (ML_OK, or the error that ended it). */
int ml_poll(ml_server *s, uint64_t job, int *done, double *out_host, size_t out_len);
/* Blocks until the request finishes (ML_ETIMEOUT after timeout_s seconds). */
int ml_wait(ml_server *s, uint64_t job, double timeout_s);
/* Host times (seconds since server creation) of submission, admission and
 * completion (-1 while not reached). */
int ml_job_times(ml_server *s, uint64_t job, double *t_submit, double *t_admit, double *t_done);
/* Forgets a finished request (ML_EBUSY while it runs). */
int ml_job_release(ml_server *s, uint64_t job);
int ml_server_stats(ml_server *s, ml_server_info *out);
/* Cancels queued requests, waits for the admitted ones, stops the worker
 * and frees everything. */
int ml_server_destroy(ml_server *s);

/* ------------------------------------------------------------------------ */
/* Allocation-free entry point (no counterpart in the paper)                  */
/* ------------------------------------------------------------------------ */

/* Some callers cannot allocate device memory: code embedded in a host
 * application or framework whose memory manager has already claimed the
 * device memory it may use (a cudaMalloc there fails or fragments its pool),
 * and latency-bound serving loops, where cudaMalloc / cudaFree may
 * synchronise the device and stall every stream.  For them this computes the
 * same values as the `naive` and `plaq` blocks of ml_observe from angles the
 * caller already holds on the device, and allocates nothing: its scratch is
 * one fixed array of ML_NOALLOC_SCRATCH_BYTES (2 MiB) inside the library,
 * which every GPU that loads the library keeps until the process exits.
 *
 *   theta_dev    device angles in the library's layout,
 *                theta[(mu * 2 + parity) * V/2 + (i >> 1)], i and parity as
 *                above; double for prec = ML_FP64, float for ML_FP32
 *   r, nr        host array of nr separations, 1 <= r <= L-1,
 *                1 <= nr <= ML_NOALLOC_MAX_R
 *   out_dev      device output, 2 nr + 1 doubles: (Re, Im) of
 *                (1/L^3) sum_x P(x)^* P(x + r xhat) for each r, then the mean
 *                plaquette
 *   cuda_stream  stream the work is enqueued on (cudaStream_t; NULL = legacy
 *                default stream); the call does not synchronise
 *
 * Size limit: a call uses 2 nr W + Wv doubles of the scratch array, with
 * W = 8 ceil(L^3 / 256) and Wv = 8 ceil(L^3 Nt / 256); a call that would need
 * more than ML_NOALLOC_SCRATCH_BYTES / 8 doubles returns ML_EINVAL (24^3 x 8
 * with nr = 11 uses 12960 of the 262144).
 * Set-up: the first call on each device looks up the device address of the
 * scratch array with that device current; make that first call before any
 * stream capture.
 * Sharing: every call on a device uses the same array and it keeps the last
 * call's contents; each call writes every value it later reads, so nothing
 * needs clearing, but calls that may overlap on the GPU (different streams
 * or host threads) race and must be serialised by the caller. */
#define ML_NOALLOC_SCRATCH_BYTES (2 * 1024 * 1024)
#define ML_NOALLOC_MAX_R 64
int ml_naive_noalloc(const void *theta_dev, int L, int Nt, int prec, const int *r, int nr, double *out_dev,
                     void *cuda_stream);

/* Static text for a status code. */
const char *ml_error_string(int status);

/* Number of kernels the library has launched in this process (including
 * those replayed from CUDA graphs). */
uint64_t ml_kernel_launches(void);

#ifdef __cplusplus
}
#endif

#endif /* ML_H */
