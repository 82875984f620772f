/*
 * fdps_gpu.h -- C ABI of a single-GPU (sm_103a) Barnes-Hut tree force for
 * softened self-gravity, shaped after the public API of FDPS
 * (Iwasawa et al. 2016, "Implementation and performance of FDPS",
 * arXiv 1601.03138).
 *
 * The paper's user program (Sect. 2.2, the N-body example) creates a
 * ParticleSystem, a TreeForForceLong object and calls
 * calcForceAllAndWriteBack(f_epj, f_spj, psys, dinfo) between a predict
 * (kick + drift) and a correct (kick) step.  This header offers the same
 * pieces as opaque handles:
 *
 *   fdps_init / fdps_finalize            <- PS::Initialize / PS::Finalize
 *   fdps_psys_*                          <- ParticleSystem<FP>
 *   fdps_tree_create                     <- TreeForForceLong<...>::Monopole
 *                                           (and the quadrupole variant)
 *   fdps_tree_calc_force_all_and_write_back
 *                                        <- calcForceAllAndWriteBack
 *   fdps_kick / fdps_drift / fdps_step   <- the example's predict/correct
 *
 * Conventions shared by every call:
 *   - Every function returning int returns FDPS_OK (0) or a negative
 *     FDPS_E* code; fdps_last_error(ctx) then holds a one-line message.
 *     No call exits the process or traps the GPU.
 *   - Handles own all their device memory; *_destroy frees it.
 *   - All work is issued on the context's CUDA stream (fdps_get_stream);
 *     calls that return data to host memory synchronise that stream.
 *   - Positions, velocities and accelerations are row-major [n][3] FP64
 *     arrays ("pos3n"); masses, softenings and potentials are [n] FP64.
 *   - Pointers flagged by on_device = 1 are device pointers borrowed for
 *     the duration of the call only; on_device = 0 means host memory.
 *   - Units: G = 1.
 */
#ifndef FDPS_GPU_H
#define FDPS_GPU_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ----------------------------------------------------------- status codes */
#define FDPS_OK 0
#define FDPS_EINVAL (-1)    /* bad argument: see fdps_last_error */
#define FDPS_ENOMEM (-2)    /* device or host allocation failed */
#define FDPS_ECUDA (-3)     /* a CUDA runtime call failed */
#define FDPS_EOVERFLOW (-4) /* an internal buffer bound was exceeded and the
                               automatic resize-and-retry also failed */
#define FDPS_ETIMEOUT (-5)  /* a bounded device-side wait gave up */
#define FDPS_ESTATE (-6)    /* call out of order (e.g. data not set yet) */

/* ------------------------------------------------------------- handles */
typedef struct fdps_ctx fdps_ctx;
typedef struct fdps_psys fdps_psys;
typedef struct fdps_tree fdps_tree;

/* --------------------------------------------------------- parameters */
enum fdps_moment { FDPS_MONOPOLE = 0, FDPS_QUADRUPOLE = 1 };
enum fdps_precision {
    FDPS_FP32REL = 0, /* walk output converted to FP32 relative to each
                         i-group's centre, FP32 force with compensated sums */
    FDPS_FP64 = 1     /* FP64 absolute coordinates and FP64 sums */
};

/* Interaction kernels selectable at run time (Sect. 2.2: the user passes one
   functor for particle-particle and one for particle-superparticle terms). */
typedef enum {
    FDPS_GRAV_EPJ = 0,      /* Eq. ParticleParticleNbody, softening eps_i */
    FDPS_GRAV_SPJ_MONO = 1, /* Eq. ParticleSuperparticleNbody (monopole) */
    FDPS_GRAV_SPJ_QUAD = 2  /* monopole + traceless quadrupole term */
} fdps_kernel_id;

/* Tree-for-force parameters (TreeForForceLong, Sect. 2.2; theta is the fixed
   opening angle of the Barnes-Hut traversal, Sect. 3.2; n_grp the group size
   of the modified tree algorithm, Sect. 5.5).
     theta      >= 0   opening angle; 0 opens every cell (direct summation)
     n_leaf     1..16  a cell with <= n_leaf particles is a leaf
     n_grp      >= n_leaf, <= 4096: a maximal cell with <= n_grp particles
                       is one i-group sharing one interaction list
     moment     enum fdps_moment
     precision  enum fdps_precision
     tile_depth list entries staged in shared memory per force-kernel chunk:
                0 (default, = 512), 256 or 512
     block      threads per CTA of the FP32 force kernel: 0 (default, =
                128), 64, 128 or 256
     i_per_thread  at most this many i-particles per thread of the FP32
                force kernel: 0 (default, = 5), 2, 4 or 5; block 256 takes
                2 at most (its Kahan sums would not fit shared memory)
     (block and i_per_thread, the "block shape", change only the speed;
     the FP64 variant ignores them)                                      */
typedef struct {
    double theta;
    int32_t n_leaf;
    int32_t n_grp;
    int32_t moment;
    int32_t precision;
    int32_t tile_depth;
    int32_t block;
    int32_t i_per_thread;
    int32_t reserved;
} fdps_tree_params;

/* Per-call counters and stage times (milliseconds, CUDA events, valid when
   profiling is on) of the last force calculation. */
typedef struct {
    int64_t n_particles;
    int64_t n_nodes;
    int64_t n_groups;
    int64_t n_levels;          /* deepest level + 1 */
    int64_t list_entries;      /* sum over groups of list entries
                                  (SPJ cells + opened leaves) */
    int64_t n_epj;             /* sum over groups of |EPJ| (particles) */
    int64_t n_spj;             /* sum over groups of |SPJ| (cells) */
    int64_t interactions_epj;  /* sum over groups of n_i |EPJ| */
    int64_t interactions_spj;  /* sum over groups of n_i |SPJ| */
    int64_t fp64_fallbacks;    /* opening tests decided in FP64 */
    int64_t retries;           /* buffer resize-and-retry count */
    int64_t sort_coherent;     /* 1: the last sort was the coherent time-step
                                  sort, 0: the radix sort */
    double ms_box_keys;        /* root box + Morton keys */
    double ms_sort;            /* sort (after the keys) */
    double ms_permute;         /* reorder into key order */
    double ms_build;           /* octree levels */
    double ms_moments;         /* bottom-up moments */
    double ms_groups;          /* i-group selection and boxes */
    double ms_walk;            /* interaction lists (after fdps_tree_neighbors:
                                  the radii's preparation and the neighbour walk) */
    double ms_force;           /* force kernel (after fdps_tree_neighbors: the
                                  pair pass) */
    double ms_total;
} fdps_tree_stats;

/* ------------------------------------------------------- PS::Initialize */

/* Select CUDA device `device`, create a stream and return a context.
   Errors: FDPS_EINVAL (no such device or not sm_103), FDPS_ECUDA. */
int fdps_init(int device, fdps_ctx** out);
/* Free the context (psys and tree handles must be destroyed first). */
int fdps_finalize(fdps_ctx* ctx);
/* Message of the last failing call on this context ("" if none). */
const char* fdps_last_error(const fdps_ctx* ctx);
/* The cudaStream_t every call is issued on (as void*). */
void* fdps_get_stream(const fdps_ctx* ctx);
/* Issue all further work on a caller-owned cudaStream_t (NULL = back to the
   context's own stream).  The caller keeps ownership. */
int fdps_set_stream(fdps_ctx* ctx, void* stream);
/* Number of CUDA kernels this library has launched on the context so far
   (-1 for NULL). */
int64_t fdps_kernel_launches(const fdps_ctx* ctx);
/* Diagnostic of the failure path of the library's one kind of device-side
   wait (the radix sort's look-back on earlier tiles, bounded to about 2^20
   polls): runs a single look-back whose predecessor never publishes.
   Returns FDPS_ETIMEOUT when the wait gave up and reported it, as designed;
   the context stays usable.  Any other result is a fault of the library. */
int fdps_selftest_bounded_wait(fdps_ctx* ctx);
/* Enable (1) / disable (0) per-stage CUDA-event timing in fdps_tree_stats. */
int fdps_set_profiling(fdps_ctx* ctx, int on);

/* ------------------------------------------------ ParticleSystem<FP> */

/* A particle system of n >= 1 particles (the example's class Nbody: mass,
   eps, pos, vel, acc, plus the potential).  Contents are undefined until
   fdps_psys_set.  Errors: FDPS_EINVAL, FDPS_ENOMEM. */
int fdps_psys_create(fdps_ctx* ctx, int64_t n, fdps_psys** out);
int fdps_psys_destroy(fdps_psys* ps);
/* getNumberOfParticleLocal: number of particles (or -1 for NULL). */
int64_t fdps_psys_size(const fdps_psys* ps);
/* Copy particle data in (the example's readAscii / copyFromFP).  pos3n and
   vel3n are [n][3]; mass [n] >= 0; eps [n] > 0 (the softening of Eq.
   ParticleParticleNbody, eps_i of the receiving particle).  vel3n may be
   NULL (zero velocities).  Values are validated on the device: NaN/Inf,
   negative mass or non-positive eps give FDPS_EINVAL.  The first data
   after fdps_psys_create or fdps_psys_set_systems, and the call after a
   rejected one, put the particles in the caller's order; later calls keep
   the order the library holds them in (the last force calculation's
   sorted order), so that a force calculation on data that moved little
   starts from nearly sorted keys.  Row i always stays particle i; the
   internal order only decides how equal Morton keys are broken
   (fdps_tree_get_keys).  on_device = 0: host arrays; the
   device reads page-locked or managed host arrays directly (over the
   CPU-GPU link, no staging copy) and stages the others through device
   memory with copies.  The call returns after the data has been read, so
   the caller may reuse its arrays at once. */
int fdps_psys_set(fdps_psys* ps, const double* pos3n, const double* vel3n,
                  const double* mass, const double* eps, int on_device);
/* Copy particle data out in the caller's order (rows as passed to
   fdps_psys_set).  Any output pointer may be NULL.  acc3n and pot are the
   results of the last force calculation (copyFromForce); the potential has
   the self term removed.  FDPS_ESTATE if acc/pot are requested before any
   force calculation.  Page-locked or managed host arrays are written by
   the device directly, others through a device staging buffer and copies;
   the call returns when the data is in place. */
int fdps_psys_get(const fdps_psys* ps, double* pos3n, double* vel3n,
                  double* acc3n, double* pot, int on_device);

/* --------------------------------------------- TreeForForceLong<...> */

/* Create a tree-for-force object (Sect. 2.2, grav.initialize).  Errors:
   FDPS_EINVAL for out-of-range parameters (see fdps_tree_params). */
int fdps_tree_create(fdps_ctx* ctx, const fdps_tree_params* params,
                     fdps_tree** out);
int fdps_tree_destroy(fdps_tree* tree);

/* calcForceAllAndWriteBack (Sect. 2.2; steps of Sect. 3.2 on one GPU):
   root box -> Morton keys -> radix sort -> reorder -> octree -> moments ->
   i-groups -> interaction lists -> forces, written back into ps
   (acceleration and potential of every particle, overwriting old values).
   k_epj must be FDPS_GRAV_EPJ; k_spj FDPS_GRAV_SPJ_MONO, or
   FDPS_GRAV_SPJ_QUAD for a quadrupole tree.  The particles are left in
   Morton order internally; fdps_psys_get still returns the caller's order.
   Errors: FDPS_EINVAL, FDPS_ESTATE (no data), FDPS_ENOMEM,
   FDPS_EOVERFLOW, FDPS_ECUDA. */
int fdps_tree_calc_force_all_and_write_back(fdps_tree* tree, fdps_psys* ps,
                                            int k_epj, int k_spj);

/* Leapfrog pieces of the example's predict/correct (Sect. 2.2):
   fdps_kick: v += dt_half * a;  fdps_drift: x += dt * v  (FP64). */
int fdps_kick(fdps_psys* ps, double dt_half);
int fdps_drift(fdps_psys* ps, double dt);
/* One kick-drift-kick step: kick(dt/2), drift(dt), force, kick(dt/2).
   Needs valid forces from a previous force calculation (FDPS_ESTATE). */
int fdps_step(fdps_tree* tree, fdps_psys* ps, double dt);
/* Kinetic sum m v^2 / 2 and potential sum m phi / 2 (FP64), using the
   potential of the last force calculation. */
int fdps_psys_energy(fdps_psys* ps, double* kinetic, double* potential);

/* ------------------------------------------------ ensembles and runs */

/* Declare the particle system an ensemble of n_sys independent systems
   (the "multiwalk" use of Sect. 2.1.2: many independent interaction sets per
   accelerator launch).  offsets is a host array [n_sys + 1] with
   offsets[0] = 0, offsets[n_sys] = n and every system holding >= 1 row:
   rows offsets[k] .. offsets[k+1]-1 of the arrays passed to fdps_psys_set
   form system k.  Every force calculation then treats each system on its
   own (its own root box, keys, octree, i-groups and lists; no system feels
   another) in the same launches.  Clears the particle data: call
   fdps_psys_set afterwards.  n_sys = 1 restores one system.
   Errors: FDPS_EINVAL (bad offsets), FDPS_ENOMEM. */
int fdps_psys_set_systems(fdps_psys* ps, int32_t n_sys, const int64_t* offsets);
/* Number of systems (1 unless set otherwise; -1 for NULL). */
int32_t fdps_psys_num_systems(const fdps_psys* ps);
/* Per-system kinetic (sum m v^2 / 2) and potential (sum m phi / 2) energy
   into host arrays [n_sys]; FDPS_ESTATE before any force calculation. */
int fdps_psys_energy_systems(fdps_psys* ps, double* kinetic, double* potential);
/* n_steps kick-drift-kick steps of the example's integrator (Sect. 2.2).
   The first step runs as fdps_step and sizes every buffer with headroom;
   each later step replays a CUDA graph of the whole step (kick, drift, the
   full force pipeline, kick) captured on the context's stream, which must
   therefore be a stream that can be captured (the context's own stream,
   or a caller stream other than the legacy default stream).  A step whose
   force calculation outgrows a captured buffer is redone with larger
   buffers and the graphs are captured again.  Needs valid forces
   (FDPS_ESTATE); synchronises the stream once per step. */
int fdps_run(fdps_tree* tree, fdps_psys* ps, double dt, int64_t n_steps);

/* Autotuner (the paper's n_grp trade-off, Sect. 5.5-5.6, measured instead
   of modelled): time the full force calculation (CUDA events, best of
   `repeats` after one untimed sizing run) for every combination of the
   candidate n_leaf, n_grp and tile_depth values at the tree's block shape
   (tile_depth may be NULL: default only); then, at the fastest of those,
   every combination of the candidate block and i_per_thread values of the
   FP32 force kernel (either may be NULL: the winner's own).  Keeps the
   fastest in the tree's parameters and leaves the forces of that choice in
   ps.  Combinations the parameter rules reject (n_grp < n_leaf, block 256
   with 4 i-particles) are skipped.  *best and *best_ms (either may be
   NULL) receive the winning parameters and its time in milliseconds.
   Theta, moment and precision are not tuned: they set the accuracy.
   Errors: FDPS_EINVAL, FDPS_ESTATE, and those of the force calculation. */
int fdps_tree_autotune(fdps_tree* tree, fdps_psys* ps, const int32_t* n_leaf, int32_t n_nl,
                       const int32_t* n_grp, int32_t n_ng, const int32_t* tile_depth,
                       int32_t n_td, const int32_t* block, int32_t n_block,
                       const int32_t* i_per_thread, int32_t n_ipt, int32_t repeats,
                       fdps_tree_params* best, double* best_ms);

/* --------------------------------------------------- introspection
   Test and diagnostic access to the last force calculation's
   intermediate data.  All outputs are host arrays; each call synchronises
   the stream.  `cap` is the capacity of every output array in elements
   (rows); FDPS_EOVERFLOW if too small.  Arrays may be NULL to skip them. */
int fdps_tree_get_stats(const fdps_tree* tree, fdps_tree_stats* out);
/* Root box {lo_x, lo_y, lo_z, L, s}: lo = per-axis minimum, L = largest
   extent (1 if 0), s = 2^21 / L. */
int fdps_tree_get_box(const fdps_tree* tree, double* out5);
/* Morton keys in the particle order the call started from, and the stable
   sort permutation (sorted position -> that order's index). */
int fdps_tree_get_keys(const fdps_tree* tree, uint64_t* keys, uint32_t* perm,
                       int64_t cap);
/* Node table in BFS order (level-major, key prefix ascending).  child_first
   is -1 for a leaf; com is [n][3]; quad [n][6] (xx yy zz xy xz yz, zero for
   a monopole tree).  *n_out receives the node count. */
int fdps_tree_get_nodes(const fdps_tree* tree, int64_t cap, int64_t* n_out,
                        int32_t* level, int64_t* first, int64_t* count,
                        int64_t* child_first, int32_t* nchild, double* mass,
                        double* com, double* quad);
/* i-groups in order of their first particle: first, count, node id and FP64
   bounding box [g][6] (lo xyz, hi xyz).  *n_out receives the group count. */
int fdps_tree_get_groups(const fdps_tree* tree, int64_t cap, int64_t* n_out,
                         int64_t* first, int64_t* count, int64_t* node,
                         double* box6);
/* Interaction lists of groups [g0, g1): offsets [g1-g0+1] into `entries`.
   An entry is a node id; bit 31 set marks an opened leaf (its particles
   are EPJ), clear marks a superparticle (SPJ).  `cap` bounds `entries`. */
int fdps_tree_get_lists(const fdps_tree* tree, int64_t g0, int64_t g1,
                        int64_t* offsets, uint32_t* entries, int64_t cap);

/* ---------------------------------------------- short-range mode
   Neighbour search over the same tree (Sect. 2.1.2, 3.2) for FDPS's four
   cutoff types, with the SPH density of the paper's SPH runs (Wendland C6
   kernel, Sect. 4.3) as the work on the neighbours.  Particle j is a
   neighbour of i (i itself included) iff r^2 < c^2, r^2 evaluated in FP64
   as (dx*dx + dy*dy) + dz*dz with each operation rounded on its own, and
     FDPS_CUTOFF_FIXED      c = r_fixed
     FDPS_CUTOFF_I          c = h_i            (gather)
     FDPS_CUTOFF_J          c = h_j            (scatter)
     FDPS_CUTOFF_SYMMETRIC  c = max(h_i, h_j)
   rho_i = sum over the neighbours of m_j W(r, H), W the 3D Wendland C6
   kernel with support H = r_fixed, h_i or h_j (symmetric: the mean of
   W(r, h_i) and W(r, h_j)), evaluated in FP32.
     h        [n] cutoff radii in the caller's order (host, or device with
              h_on_device = 1); ignored (may be NULL) for the fixed type
     counts   [n] neighbour counts, rho [n] densities, in the caller's order
              (host, or device with out_on_device = 1); either may be NULL
     info3    optional host [3]: neighbour pairs, candidate pairs tested,
              pairs decided by the FP64 sequence
   The tree's n_leaf and n_grp apply; the tree's lists afterwards hold the
   neighbour candidates (opened leaves), not gravity lists.  Synchronous.
   Errors: FDPS_EINVAL (type, radius, NULL radii, non-positive radii),
   FDPS_ESTATE, FDPS_ENOMEM, FDPS_EOVERFLOW, FDPS_ECUDA. */
#define FDPS_CUTOFF_FIXED 0
#define FDPS_CUTOFF_I 1
#define FDPS_CUTOFF_J 2
#define FDPS_CUTOFF_SYMMETRIC 3
int fdps_tree_neighbors(fdps_tree* tree, fdps_psys* ps, int32_t mode, double r_fixed,
                        const double* h, int h_on_device, uint32_t* counts, double* rho,
                        int out_on_device, int64_t* info3);

/* ------------------------------------------ accuracy diagnostics
   fdps_direct_sample: the exact reference of the force law (Eq.
   ParticleParticleNbody summed over every other particle of the same
   system, softening of the receiving particle) for n_sample particles
   given by their rows in the caller's arrays (host array `rows`, values in
   0 .. n-1).  Arithmetic: separations from FP32 hi/lo position parts (about
   48 bits), FP32 pair terms, compensated sums finished in FP64 (relative
   error about 1e-6 or below).  acc3 [n_sample][3] and pot [n_sample] are
   host outputs (either may be NULL).  Synchronous.  Errors: FDPS_EINVAL,
   FDPS_ESTATE (no data), FDPS_ENOMEM, FDPS_ECUDA.

   fdps_tree_choose_theta: the largest opening angle among `candidates`
   (n_candidates values; NULL: 0.2, 0.3, ..., 1.0) whose median relative
   acceleration error |a_tree - a_direct| / |a_direct| over n_sample evenly
   spaced rows stays at or below `target`.  It tries the candidates in
   increasing order with full force calculations, stops at the first that
   misses the target, sets the tree's theta to the choice (the smallest
   candidate if none meets the target) and leaves the forces of that
   choice in ps.  *theta_out and *median_out (either may be NULL) receive
   the choice and its measured median.  Errors as for the force
   calculation and fdps_direct_sample. */
int fdps_direct_sample(fdps_psys* ps, int64_t n_sample, const int64_t* rows,
                       double* acc3, double* pot);
int fdps_tree_choose_theta(fdps_tree* tree, fdps_psys* ps, double target,
                           int64_t n_sample, const double* candidates,
                           int32_t n_candidates, double* theta_out, double* median_out);

/* --------------------------------------- user interaction kernels
   FDPS takes the interaction law as user functors (Sect. 2.2: the EPJ and
   SPJ force kernels passed to calcForceAllAndWriteBack).  A C ABI cannot
   take a device functor, so user laws are compiled by the user against
   the header template fdps_user_force.cuh, which walks the lists described
   by a view.

   fdps_tree_build_lists runs the force calculation up to and including
   the interaction lists (root box, keys, sort, reorder, octree, moments,
   i-groups, lists) and computes no force.  Errors as for
   fdps_tree_calc_force_all_and_write_back.

   fdps_tree_get_view fills *view with device pointers into the tree's
   buffers for the lists of `ps` (built by either call above).  They stay
   valid until the next call that rebuilds the tree or destroys it or `ps`;
   kick or drift do not move the copies the view points to.  Layouts (all
   device memory, owned by the library, read only; float4 = 4 consecutive
   floats, 16-byte aligned):
     g_first, g_count  [n_groups] first sorted position and size of group g
     g_off, g_len      [n_groups] list of g = pool[g_off[g] .. + g_len[g])
     g_ch, g_cl        [n_groups] float4: group centre relative to the
                       system's root centre c0 as FP32 hi and lo parts
     pool              list entries: a node id; (id | leaf_tag) marks an
                       opened leaf, whose particles are EPJ; else an SPJ
     nd_first, nd_count  [nodes] first sorted position and size of a node
     nd_f              [2 nodes] float4: (COM hi - c0, M), (COM lo, 0)
     nd_fq0, nd_fq1    [nodes] float4 (Qxx, Qyy, Qzz, Qxy) and float2
                       (Qxz, Qyz): traceless quadrupole about the COM
                       (NULL for a monopole tree)
     pf_hi, pf_lo      [n] float4: (x hi - c0, y hi, z hi, m) and
                       (x lo, y lo, z lo, eps^2) of sorted particle p
     id                [n] sorted position -> the caller's row
   A position relative to a group centre is (hi - ch) + (lo - cl) per axis.
   Errors: FDPS_EINVAL (NULL, FP64-precision tree), FDPS_ESTATE (no lists
   of ps), FDPS_ECUDA. */
typedef struct {
    int64_t n;
    int64_t n_groups;
    int32_t quadrupole;
    uint32_t leaf_tag;
    const uint32_t* g_first;
    const uint32_t* g_count;
    const unsigned long long* g_off;
    const uint32_t* g_len;
    const float* g_ch;
    const float* g_cl;
    const uint32_t* pool;
    const uint32_t* nd_first;
    const uint32_t* nd_count;
    const float* nd_f;
    const float* nd_fq0;
    const float* nd_fq1;
    const float* pf_hi;
    const float* pf_lo;
    const uint32_t* id;
} fdps_tree_view;
int fdps_tree_build_lists(fdps_tree* tree, fdps_psys* ps);
int fdps_tree_get_view(const fdps_tree* tree, const fdps_psys* ps, fdps_tree_view* view);

/* User laws from source text, compiled at run time (NVRTC, sm_103a).
   `source` is CUDA C++ defining
     struct Force { ...; __device__ void clear(); };   (trivially copyable)
     struct Law   { the two __device__ call operators of
                    fdps_user_force.cuh, for Epj and for Spj tiles };
   with Epi, Epj, Spj and the rest of that header in scope; it is compiled
   together with the header's device part as the library was built.
   fdps_user_law_compile: on success *law is a handle owned by the caller
   (fdps_user_law_destroy); on a compile error it returns FDPS_EINVAL and
   the compiler's messages, with line numbers of `source`, go to `log`
   (log_cap bytes, NUL-terminated; NULL for none), as they also do on
   success (warnings).  FDPS_ECUDA if the result cannot be loaded.
   fdps_user_law_force_size: sizeof(Force) as compiled, -1 for NULL.
   fdps_user_law_run: queues the law over the lists of `ps` (built by
   fdps_tree_build_lists or a force calculation) on the context's stream;
   `out` is a device array of n Force values, out[row] for the caller's
   row `row`.  Errors as fdps_tree_get_view, and FDPS_ECUDA. */
typedef struct fdps_user_law fdps_user_law;
int fdps_user_law_compile(fdps_ctx* ctx, const char* source, fdps_user_law** law,
                          char* log, int64_t log_cap);
int64_t fdps_user_law_force_size(const fdps_user_law* law);
int fdps_user_law_run(fdps_user_law* law, const fdps_tree* tree, const fdps_psys* ps,
                      void* out);
int fdps_user_law_destroy(fdps_user_law* law);

/* ------------------------------------------- allocation-free key sort
   The paper has no counterpart to this call; it is a service for callers
   that may not allocate device memory themselves: hosts such as frameworks
   that hand out all device memory through their own pool allocator, and
   real-time loops that may not take the implicit synchronisation and
   unbounded latency of a cudaMalloc / cudaFree.  It computes what
   fdps_tree_calc_force_all_and_write_back
   computes first (root box, 63-bit Morton keys, stable radix sort) for one
   particle set and allocates nothing: its scratch (about 5.3 MB) is a
   file-scope device array that every GPU which loads the library holds
   until the process exits.
     x, y, z      device arrays of n FP64 positions (SoA), borrowed
     n            1 .. FDPS_NOALLOC_MAX_N; larger n returns FDPS_EINVAL
     keys_sorted  device output [n]: the keys in ascending order
     perm         device output [n]: sorted position -> input index (ties
                  keep input order)
     stream       cudaStream_t to run on (NULL = legacy default stream)
   Returns FDPS_OK, FDPS_EINVAL (NULL pointer, n out of range) or
   FDPS_ECUDA (also when a CUDA error was already pending on the calling
   thread; that error is left pending for the caller).  The work is queued
   on `stream` and not waited for.  The first call on a device, with that
   device current, looks up the scratch array's device address and keeps it
   for the process.  The address belongs to the device's primary context (the one the CUDA
   runtime API uses): calls from other contexts, or after a cudaDeviceReset
   of the device, are not supported.  All calls on a device share the one
   scratch array, which keeps the last call's contents: calls that may
   overlap on the GPU (other streams, other host threads) race and must be
   serialised by the caller. */
#define FDPS_NOALLOC_MAX_N (1 << 18)
int fdps_morton_sort_noalloc(const double* x, const double* y, const double* z,
                             int64_t n, uint64_t* keys_sorted, uint32_t* perm,
                             void* stream);

#ifdef __cplusplus
}
#endif
#endif /* FDPS_GPU_H */
