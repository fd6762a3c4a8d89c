/*
 * treepm_sr.h -- C-ABI of libtreepm_sr.so, the GB300 (sm_103a) short-range
 * TreePM gravity path of Ishiyama, Nitadori & Makino (SC12).
 *
 * Problem statement (Sec. II, Eq. 2): given periodic positions r_i in the unit
 * box, masses m_i and the gravitational constant G, return for every particle
 * the short-range acceleration
 *
 *     f_i = sum_{j != i} G m_j (r_j - r_i) / (|r_j - r_i|^2 + eps^2)^{3/2}
 *                        * g_P3M(2 |r_j - r_i| / r_cut)                 (Eq. 2)
 *
 * with the cutoff shape g_P3M of Eq. 3 (zero for |r_j - r_i| >= r_cut), the
 * minimum-image convention of the periodic box (Sec. I), and the sum evaluated
 * with Barnes' grouped tree traversal (Sec. II): each group of nearby particles
 * shares one interaction list of particles and monopole tree nodes, built by a
 * cutoff-pruned walk with opening angle theta (Sec. I).  Eq. 2 carries no m_i:
 * the result is an acceleration.
 *
 * Conventions common to every call
 *   - Pointers marked "device" must be CUDA device (or managed) memory of the
 *     current device; pointers marked "host" are ordinary host memory.
 *   - stream is a cudaStream_t passed as void* (NULL = the legacy default
 *     stream).  Work is enqueued on it; calls return without waiting unless
 *     stated otherwise.  A tree also owns a second (non-blocking) stream on
 *     which the builds run the steps that do not depend on each other; it
 *     forks from and joins back into `stream` by events within each call, so
 *     the work stays ordered on `stream` and captures into one graph.
 *   - Positions are FP64 [n][3] row-major (x,y,z per particle), any finite
 *     value (they are wrapped into [0,1)).  Masses are FP64 [n] >= 0, or NULL
 *     for equal masses 1/n.
 *   - The caller owns every buffer it passes; they must stay valid until the
 *     enqueued work has completed.  The library owns tp_tree and everything it
 *     allocates, released only by tp_tree_free.
 *   - Errors are returned, never raised: no call aborts, exits or throws.
 *     Argument errors return synchronously.  Errors detected on the device
 *     (list overflow, non-finite positions, a bounded wait that expired) are
 *     latched in the tree and returned by tp_tree_status and by the next call
 *     on that tree that synchronises.
 */
#ifndef TREEPM_SR_H
#define TREEPM_SR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    TP_OK = 0,
    TP_ERR_INVALID_ARG = -1,   /* a bad pointer, size or parameter           */
    TP_ERR_CUDA = -2,          /* a CUDA runtime call failed                 */
    TP_ERR_OOM = -3,           /* device allocation failed                   */
    TP_ERR_LIST_OVERFLOW = -4, /* a preallocated capacity was too small      */
    TP_ERR_TIMEOUT = -5,       /* a bounded device-side wait expired         */
    TP_ERR_NONFINITE = -6,     /* a position was NaN or infinite             */
    TP_ERR_NO_DEVICE = -7      /* no usable CUDA device                      */
} tp_status;

typedef enum { TP_FP64 = 0, TP_FP32 = 1 } tp_precision;

/* Per-box parameters (Sec. II and III-A).
 *   G       gravitational constant
 *   eps     Plummer softening length, 0 <= eps (Sec. II: eps << r_cut)
 *   r_cut   cutoff radius, 0 < r_cut < 0.5 of the unit box (Sec. III-A uses
 *           r_cut = 3 / N_PM^{1/3})
 *   theta   opening angle, >= 0; 0 gives the exact cutoff sum
 *   n_crit  largest group size (Barnes' modified algorithm, Sec. II), 1..4096
 *   n_leaf  a tree node holding more than n_leaf particles is split, 1..64
 *   precision  TP_FP32 (pair arithmetic in FP32 on group-relative
 *           coordinates) or TP_FP64 (plain FP64 reference path)
 *   flags   0, or any of TP_FLAG_CHUNKED, TP_FLAG_XI_SOFTENED and
 *           TP_FLAG_RSQRT_REFINED                                           */
typedef struct {
    double G, eps, r_cut, theta;
    int32_t n_crit, n_leaf, precision, flags;
} tp_params;

/* Bounded list memory (a property of this implementation; the paper builds
 * each group's list as it goes).  Normally every group's interaction list is
 * kept on the device (20 bytes per entry).  In chunked mode the walk and the
 * pair kernels run over windows of consecutive groups whose lists fit a fixed
 * budget of 2^29 entries (about 11 GB), so a box whose lists would not fit in
 * device memory can still be evaluated; the lists are not kept between calls
 * (tp_export_lists returns TP_ERR_INVALID_ARG), every force/vjp call re-walks
 * each window, and a force/vjp call after tp_rebuild_tree synchronises the
 * stream once to plan the windows (so it cannot be captured in a CUDA graph).
 * The build switches to chunked mode by itself when whole lists (24 bytes per
 * padded slot of the walk) would take more than half of the device memory
 * that is free at build time; setting TP_FLAG_CHUNKED in any box's flags
 * forces it (with windows of about a quarter of the lists, which also
 * exercises the mode on small boxes).  Results are the same as with whole
 * lists.  tp_tree_stats reports n_windows > 1 for a chunked tree.           */
#define TP_FLAG_CHUNKED 1

/* Cutoff argument from the softened distance (the paper's kernel form, Sec.
 * II-A, which takes one inverse square root per pair for both the softened
 * 1/s^3 factor and the cutoff argument).  By default a pair at distance r
 * contributes G m_j d g(2r/r_cut) / (r^2 + eps^2)^{3/2} and vanishes for
 * r >= r_cut.  With this flag the cutoff argument is 2s/r_cut with
 * s = sqrt(r^2 + eps^2): a pair contributes G m_j d g(2s/r_cut) / s^3 and
 * vanishes for s >= r_cut.  The two differ by O(eps^2 / r_cut^2) relative.
 * The lists (cut at r_cut) are the same.  All boxes of a batched tree must
 * agree on this flag (else TP_ERR_INVALID_ARG).  tp_short_range_vjp and
 * tp_short_range_force_vjp differentiate the variant the tree was built
 * with.  tp_short_range_force_noalloc does not take it.                    */
#define TP_FLAG_XI_SOFTENED 2

/* The paper's inverse square root (Sec. II-A) in the FP32 pair kernels: 1/s
 * from an estimate y0 refined by one third-order step, h0 = 1 - x y0^2 and
 * y1 = y0 (1 + h0/2 + 3 h0^2/8), instead of the hardware reciprocal square
 * root.  The paper's processor has an 8-bit estimate instruction; here the
 * estimate is Lomont's integer approximation (the FP32 bit pattern of x
 * shifted right by one and subtracted from 0x5f3759df) after one Newton
 * step, off by less than 1.8e-3, so y1 is good to about 1.5e-8.  It moves
 * the root from the MUFU pipe to about ten FP32 operations on the FMA pipe
 * (the pipe that bounds these kernels, so it is slower on GB300).  FP32 trees
 * only (else TP_ERR_INVALID_ARG); the kernels for groups spanning half the
 * box or with eps = 0 keep the hardware root.  All boxes of a batched tree
 * must agree on this flag.                                                  */
#define TP_FLAG_RSQRT_REFINED 4

typedef struct tp_tree tp_tree; /* opaque, library-owned */

/* Statistics of a built tree (Table I reports the same quantities).
 * n_interactions = sum over groups of n_i * n_j, the paper's count of the
 * pairs the force loop evaluates (Sec. III-B).  n_useful = how many of those
 * pairs have a non-zero Eq. 2 term: a positive distance r and a cutoff
 * distance (r, or sqrt(r^2 + eps^2) with TP_FLAG_XI_SOFTENED) below r_cut,
 * decided in FP64 from the FP64 positions and centres of mass; counted by a
 * pass over the lists on each tp_tree_stats call (about a quarter of a force
 * call's time), -1 for a tree in chunked mode (its lists are not kept).  In
 * chunked mode the list quantities are those of the last build or force
 * call.                                                                     */
typedef struct {
    int64_t n, n_nodes, n_groups, n_entries, n_interactions;
    int64_t n_useful;      /* evaluated pairs inside the cutoff (see above)  */
    int64_t n_ambiguous;   /* walk decisions settled by the exact FP64 test  */
    double mean_ni, mean_nj;
    int32_t max_nj, nbox;
    int64_t n_windows;     /* group windows of chunked mode; 1 otherwise     */
} tp_stats;

/* Build the tree of one box: Morton keys, sort, octree, monopoles, groups
 * and interaction lists (Sec. I and II).  pos: device [n][3]; mass: device
 * [n] or NULL; p: host.  Synchronises `stream` once (sizes are read back) and
 * returns the first error seen, including device-detected ones.  On success
 * *out receives a new tree (free it with tp_tree_free).  n = 0 is valid.     */
tp_status tp_build_tree(const double *pos, const double *mass, int64_t n,
                        const tp_params *p, void *stream, tp_tree **out);

/* The same for nbox independent periodic unit boxes stored back to back:
 * box b holds particles [box_offsets[b], box_offsets[b+1]) of pos/mass.
 * box_offsets: host [nbox+1], non-decreasing, box_offsets[0] = 0.
 * per_box: host [nbox], one parameter set per box (precision must agree).
 * Forces and gradients of a batched tree are written for all boxes at once,
 * in the input order of pos.                                                */
tp_status tp_build_tree_batched(const double *pos, const double *mass,
                                const int64_t *box_offsets, int32_t nbox,
                                const tp_params *per_box, void *stream, tp_tree **out);

/* Rebuild an existing tree in place from new positions (same n, boxes and
 * parameters) without allocating and without synchronising: every size is
 * kept on the device, so the call can be captured in a CUDA graph.  If a
 * capacity taken from the previous build is exceeded, TP_ERR_LIST_OVERFLOW is
 * latched (check tp_tree_status after the work completes) and the following
 * force/vjp calls write zeros; rebuild outside the graph with tp_build_tree. */
tp_status tp_rebuild_tree(tp_tree *t, const double *pos, const double *mass, void *stream);

/* Keep the tree's structure, groups and interaction lists from its last
 * (re)build and refresh everything that depends on positions: the particle
 * images, the node monopoles (mass, centre of mass, box) and the list entries'
 * FP32 records.  For integrators that reuse the lists over several short
 * steps -- the paper's multiple-stepsize scheme evaluates the PP part more
 * often than the PM part -- and for derivatives with a frozen tree.
 * pos: device [n][3], the same particles in the same order as the build;
 * each is taken at the periodic image nearest to its position at the last
 * build, so displacements must stay below half the box (and, for the lists to
 * stay complete, well below r_cut: entries are neither added nor removed,
 * pairs beyond r_cut still contribute exactly zero).  mass: device [n] or NULL
 * to keep the masses.  No allocation, no synchronisation (graph-capturable).
 * TP_ERR_INVALID_ARG for a tree in chunked mode (its lists are not kept).   */
tp_status tp_refit_tree(tp_tree *t, const double *pos, const double *mass, void *stream);

/* Short-range accelerations, Eq. 2, for the lists of t.  acc: device [n][3]
 * in input order; float when the tree's precision is TP_FP32, double when it
 * is TP_FP64.  Overwritten.  Asynchronous.                                  */
tp_status tp_short_range_force(tp_tree *t, void *acc, void *stream);

/* Vector-Jacobian product of tp_short_range_force for the fixed tree and
 * lists of t: given cot = dL/da (device [n][3], same type as acc), writes
 * grad = dL/dx (device [n][3] double, input order, overwritten).  Per pair
 * the 3x3 tidal tensor J = phi I + (phi'/r) d d^T of Eq. 2's term acts on the
 * cotangent; monopole entries pass their share to member particles through
 * the centre of mass.  Walk decisions are piecewise constant and are not
 * differentiated.  Asynchronous.                                            */
tp_status tp_short_range_vjp(tp_tree *t, const void *cot, double *grad, void *stream);

/* The force of tp_short_range_force and the vector-Jacobian product of
 * tp_short_range_vjp in one pass over the lists (no counterpart in the paper).
 * For callers that know the cotangent before they need the forces: a loss
 * linear in the accelerations, or the backward pass of a leapfrog step, where
 * a step's force is recomputed next to its VJP.  The FP32 path's adjoint
 * kernel already evaluates m_j g / s^3 for every pair and adds the Eq. 2 sum
 * per particle alongside; an FP64 tree runs the two calls in turn.  acc:
 * device [n][3] (float for TP_FP32, double for TP_FP64), cot: device [n][3]
 * of the same type, grad: device double [n][3]; all input order,
 * overwritten.  Results agree with the separate calls within rounding (the
 * particle-side sums are taken in a different order).  Asynchronous.        */
tp_status tp_short_range_force_vjp(tp_tree *t, void *acc, const void *cot, double *grad, void *stream);

/* Synchronise the tree's last stream and return its first latched error.   */
tp_status tp_tree_status(tp_tree *t);

/* Host copy of the tree statistics (synchronises).                          */
tp_status tp_tree_stats(tp_tree *t, tp_stats *out);

/* Parity exports (synchronise; host buffers sized from tp_tree_stats).
 * keys: [n] Morton keys in key order; perm: [n] input index of each sorted
 * particle.                                                                 */
tp_status tp_export_keys(tp_tree *t, uint64_t *keys, int64_t *perm);
/* ints: [n_nodes][7] = level, first, count, first_child (-1 leaf), n_children,
 * parent (-1 root), box; dbl: [n_nodes][16] = M, com xyz, lo xyz, hi xyz,
 * centre xyz, half-width xyz.  Nodes are numbered breadth first.            */
tp_status tp_export_nodes(tp_tree *t, int64_t *ints, double *dbl);
/* ints: [n_groups][3] = first, count, box; dbl: [n_groups][6] = centre xyz,
 * half-width xyz.                                                           */
tp_status tp_export_groups(tp_tree *t, int64_t *ints, double *dbl);
/* offsets: [n_groups+1]; entries: [n_entries], >= 0 a particle (key-order
 * index), < 0 a node -(id+1); each group's list in depth-first order.       */
tp_status tp_export_lists(tp_tree *t, int64_t *offsets, int32_t *entries);

/* Releases the tree and all its device memory.  Synchronises the stream of
 * the tree's last call first, so work still in flight finishes; clears any
 * pending CUDA error.  The handle is invalid afterwards; NULL is a no-op.
 * Always TP_OK.                                                             */
tp_status tp_tree_free(tp_tree *t);

/* Tile shape of the FP32 pair kernels, a tuning knob with no counterpart in
 * the paper: group particles per thread of the forward kernel (1, 2 or 4) and
 * list entries per thread of the adjoint kernel (2 or 4; or 8, held as four
 * pairs of entries in the f32x2 operations of the forces-and-adjoint pass,
 * with 4 for the adjoint alone); 2 and 4 by default.
 * Applies to later force / vjp calls on t (not to calls already enqueued).
 * Results agree to rounding (the per-particle sums are taken in a different
 * order).  TP_ERR_INVALID_ARG for other values.                              */
tp_status tp_tree_set_tile(tp_tree *t, int32_t fwd_particles, int32_t adj_entries);

/* Kernel timing, a measurement aid with no counterpart in the paper.  With
 * enable != 0 the tree records CUDA events on the call's stream immediately
 * before and after its main FP32 pair-kernel launch in tp_short_range_force
 * and its main FP32 adjoint-kernel launch in tp_short_range_vjp and
 * tp_short_range_force_vjp (the kernels that handle the groups not spanning
 * half the box, with eps > 0; not in chunked mode).  Creates the events on
 * first use (TP_ERR_CUDA if that fails).  enable = 0 stops the recording.   */
tp_status tp_tree_set_kernel_timing(tp_tree *t, int32_t enable);
/* Failure injection for tests (no counterpart in the paper): caps the node
 * visits of every walk of later builds at `budget` (0 restores the default,
 * n_nodes + 1, which a depth-first walk over skip pointers never exceeds).
 * A walk that runs out ends its list there and latches TP_ERR_TIMEOUT,
 * which tp_tree_status and the next call return; nothing waits or faults.
 * budget < 0: TP_ERR_INVALID_ARG.                                           */
tp_status tp_tree_set_walk_budget(tp_tree *t, int64_t budget);

/* Durations in ms of those two launches in the last force and vjp calls made
 * with timing on; -1 for a call that recorded nothing (timing off, FP64 tree,
 * n = 0).  Synchronises on the events.  The events are recorded as external
 * events, so calls captured in a CUDA graph with timing on time the kernels
 * of each replay (read after the replay).                                   */
tp_status tp_tree_kernel_ms(tp_tree *t, double *force_ms, double *vjp_ms);

/* Largest particle count tp_short_range_force_noalloc accepts.              */
#define TP_NOALLOC_MAX_N 65536

/* Short-range accelerations of one small box without allocating device
 * memory.  This entry point has no counterpart in the paper: it exists for
 * callers that must not let a library call cudaMalloc -- an application whose
 * device memory is carved from its own pool, or a latency-critical loop that
 * cannot afford an allocation's implicit synchronisation.  Its scratch (the
 * particles' fixed-point images and masses, 28 bytes per particle, and a
 * status word) is one statically sized device array of TP_NOALLOC_MAX_N
 * entries (1.8 MB), which every GPU that loads the library holds until the
 * process exits.  It computes the exact cutoff sum over all pairs: the same
 * force as tp_build_tree + tp_short_range_force at theta = 0, up to FP32
 * rounding.
 *   pos   device FP64 [n][3], memory of the current device (or managed)
 *   mass  device FP64 [n] or NULL (every mass 1/n)
 *   n     0 <= n <= TP_NOALLOC_MAX_N, else TP_ERR_INVALID_ARG
 *   p     host; precision must be TP_FP32 and flags 0, 0 < r_cut < 0.5,
 *         eps >= 0, G finite (else TP_ERR_INVALID_ARG); theta, n_crit and
 *         n_leaf are not used
 *   acc   device FP32 [n][3], input order, overwritten
 * A NaN or infinite position returns TP_ERR_NONFINITE and leaves acc
 * unwritten: to return it, the call synchronises `stream` once, after the
 * positions are converted and before the pair sum is enqueued.  The pair sum
 * itself is asynchronous.  The first call on a device looks up the array's
 * device address (once per device, with that device current) and keeps it
 * for the life of the process; a cudaDeviceReset invalidates it, so do not
 * call this entry point after one.  Every call rewrites the scratch it reads,
 * so nothing needs clearing, but all calls share the one array: calls that
 * overlap on the GPU (on different streams, or from different threads) race. */
tp_status tp_short_range_force_noalloc(const double *pos, const double *mass, int64_t n,
                                       const tp_params *p, float *acc, void *stream);

/* ------------------------------------------------------------------------
 * The long-range (PM) half of TreePM (Sec. II, cycle of Sec. II-B).  Each tp_pm_force call runs
 * the PM cycle on one GPU over an n_mesh^3 periodic mesh of the unit box
 * (mesh point (i,j,k) at (i,j,k)/n_mesh):
 *   1. TSC assignment of the masses to the 27 mesh points around each
 *      particle's nearest one;
 *   2. FFT, product with the Green's function of the long-range force, and
 *      the inverse FFT, which give the potential on the mesh;
 *   3. -grad(phi) on the mesh by the four-point finite difference;
 *   4. TSC interpolation of that mesh force to each particle.
 * The long-range pair force is the force between two S2 clouds of radius
 * r_cut/2 (Eq. 1), the complement of the cutoff g_P3M of Eq. 3, so that
 * tp_short_range_force + tp_pm_force with the same r_cut and G is the whole
 * TreePM acceleration.  Green's function: -4 pi G S(k)^2 / k^2, with
 * S(x) = 12 (2 - 2 cos x - x sin x) / x^4 at x = |k| r_cut / 2.  It is
 * divided by the square of the TSC window prod_a sinc(k_a h/2)^3 (for the
 * assignment and the interpolation) and is 0 at k = 0, which removes the
 * mean density as a periodic Ewald sum does.  The mesh, the FFTs (cuFFT) and
 * the interpolation are FP32.  The paper takes r_cut = 3 / n_mesh (three
 * mesh spacings).  eps does not enter the PM part.                          */
typedef struct tp_pm tp_pm; /* opaque, library-owned */

/* Allocates the mesh (36 bytes per cell: the FP32 mass/potential mesh, the
 * FP32 force mesh as float4, the half spectrum and the Green's table), the
 * two cuFFT plans and the Green's table (computed on `stream`, which is
 * synchronised once).
 *   n_mesh  even, 8 <= n_mesh <= 1024
 *   r_cut   0 < r_cut < 0.5, the same as the short-range half's
 *   G       finite
 * Errors: TP_ERR_INVALID_ARG, TP_ERR_NO_DEVICE, TP_ERR_OOM, TP_ERR_CUDA.     */
tp_status tp_pm_create(int32_t n_mesh, double r_cut, double G, void *stream, tp_pm **out);

/* Long-range accelerations of n particles.
 *   pos   device FP64 [n][3], any finite values (wrapped into the box)
 *   mass  device FP64 [n] or NULL (every mass 1/n)
 *   acc   device FP32 [n][3], input order; overwritten, or added to when
 *         accumulate != 0 (e.g. onto tp_short_range_force's output)
 * Asynchronous on `stream`.  One tp_pm serves one stream at a time.         */
tp_status tp_pm_force(tp_pm *pm, const double *pos, const double *mass, int64_t n, float *acc,
                      int32_t accumulate, void *stream);

/* The adjoint of tp_pm_force: dL/dx of L = sum_i cot_i . a_i (positions in
 * input order), through the TSC interpolation and the TSC assignment:
 *   dL/dx_k = sum_c grad W_k(c) [cot_k . A(c) + m_k B(c)],
 * A the mesh force, B = K div(U) with U the TSC assignment of the cotangent
 * vectors, div the four-point divergence and K the potential solve (FFT,
 * Green's function, FFT^-1).  The masses are held fixed.
 *   cot   device FP32 [n][3] = dL/da
 *   grad  device FP64 [n][3]; overwritten, or added to when accumulate != 0
 *         (e.g. onto tp_short_range_vjp's output)
 * The first adjoint call on a tp_pm allocates 16 more bytes per mesh cell
 * (make it before any stream capture).  Asynchronous.                      */
tp_status tp_pm_vjp(tp_pm *pm, const double *pos, const double *mass, int64_t n, const float *cot,
                    double *grad, int32_t accumulate, void *stream);

/* tp_pm_force and tp_pm_vjp in one call: the mesh force of the positions
 * is computed once.  accumulate applies to both acc and grad.               */
tp_status tp_pm_force_vjp(tp_pm *pm, const double *pos, const double *mass, int64_t n, float *acc,
                          const float *cot, double *grad, int32_t accumulate, void *stream);

/* Copies a mesh of the last call to host memory (synchronous): which = 0 the
 * potential [n_mesh^3] (after tp_pm_vjp or tp_pm_force_vjp: the adjoint's B
 * instead), which = 1 the mesh acceleration -grad(phi) [n_mesh^3][3]; layout
 * (i n_mesh + j) n_mesh + k.                                                */
tp_status tp_pm_export_mesh(tp_pm *pm, int32_t which, float *host);

/* Releases the mesh and plans (synchronises the device).  NULL is a no-op.  */
tp_status tp_pm_free(tp_pm *pm);

/* ------------------------------------------------------------------------
 * Spatial decomposition of one box over several GPUs (Sec. II: the box is cut
 * into rectangular domains by a 3-D multi-section decomposition, one per
 * process; each process evaluates the short-range forces on the particles of
 * its domain).  Because the short-range force vanishes beyond r_cut, a
 * domain needs, besides its own particles, only the particles within r_cut of
 * its box ("ghosts"; the paper's processes exchange tree data for the same
 * reason).  A tp_halo holds one geometry and selects, on the device, which
 * particles go where:
 *   - owner selection: every particle to the domain that holds it (the
 *     particle exchange after the domains move);
 *   - ghost selection: every particle of domain `self` to every other domain
 *     whose box lies within r_cut of it, periodic distance.
 * The tree, the walk and the pair kernels then run unchanged on each
 * process's own particles followed by its ghosts (the forces on the ghosts
 * are discarded, and their share of the adjoint goes back to their owners).
 * The collectives themselves (variable all-to-all) belong to the caller.
 *
 * Geometry: nx slabs along x cut at xc[0..nx]; slab i is cut into ny columns
 * at yc[i][0..ny]; column (i, j) into nz cells at zc[i][j][0..nz].  Domain
 * d = (i ny + j) nz + k is the half-open box [xc[i], xc[i+1]) x
 * [yc[i][j], yc[i][j+1]) x [zc[i][j][k], zc[i][j][k+1]).  Every list of cuts
 * starts at 0, ends at 1 and is non-decreasing.  Positions are wrapped into
 * [0,1) first, as the tree does.  Decisions are FP64 with every operation
 * rounded separately: the owner by the largest cut <= the coordinate, the
 * ghost test by the squared periodic point-to-box distance < r_cut^2, the
 * per-axis distance being 0 inside the box and otherwise the shorter of
 * (lo - p) and (p + 1) - hi when p < lo, of (p - hi) and (lo + 1) - p when
 * p >= hi.  (No counterpart in the paper for the interface itself.)       */
#define TP_MAX_DOMAINS 4096
#define TP_HALO_OWNER 0
#define TP_HALO_GHOSTS 1
typedef struct tp_halo tp_halo; /* opaque, library-owned */

/* A geometry of nx x ny x nz domains (1 <= nx ny nz <= TP_MAX_DOMAINS),
 * without cuts yet.  Allocates a few device buffers.                        */
tp_status tp_halo_create(int32_t nx, int32_t ny, int32_t nz, tp_halo **out);

/* Sets the cuts: xc host [nx+1], yc host [nx][ny+1], zc host [nx][ny][nz+1]
 * (layout above).  TP_ERR_INVALID_ARG unless every list starts at 0, ends at
 * 1 and is non-decreasing.  Synchronous (copies to the device).            */
tp_status tp_halo_set_cuts(tp_halo *h, const double *xc, const double *yc, const double *zc);

/* Selects particles of pos (device FP64 [n][3], finite) for each domain:
 * mode TP_HALO_OWNER (self and r_cut ignored) or TP_HALO_GHOSTS (0 <= self <
 * ndom, 0 < r_cut < 0.5).  Writes the selected particle indices to idx
 * (device int32 [cap]) grouped by destination domain, domain 0 first, in
 * ascending order within each destination, and the number per destination
 * to counts (host int64 [nx ny nz]).  Synchronises `stream` once.  Returns
 * TP_ERR_LIST_OVERFLOW when the total exceeds cap (counts are still filled:
 * call again with a larger idx; cap = 0 only counts), TP_ERR_NONFINITE for a
 * NaN or infinite position.  The count scratch grows with n (allocation).   */
tp_status tp_halo_select(tp_halo *h, const double *pos, int64_t n, int32_t mode, int32_t self, double r_cut,
                         int32_t *idx, int64_t cap, int64_t *counts, void *stream);

/* Releases the halo (synchronises the device).  NULL is a no-op.            */
tp_status tp_halo_free(tp_halo *h);

/* Row gather for packing exchange buffers: dst[r] = src[idx[r]] for rows of
 * `words` 32-bit words (FP64 positions: 6, FP64 masses or int64 ids: 2, FP32
 * 3-vectors: 3); all device; m rows.  Asynchronous.                         */
tp_status tp_gather_rows(const void *src, int32_t words, const int32_t *idx, int64_t m, void *dst, void *stream);

/* Scatter-add of FP64 rows of `width` values: dst[idx[r]] += src[r] (device;
 * FP64 atomics, so repeated indices sum in an unspecified order).  For
 * returning the ghosts' share of the adjoint to their owners.  Asynchronous. */
tp_status tp_scatter_add_rows(double *dst, int32_t width, const int32_t *idx, const double *src, int64_t m,
                              void *stream);

/* Leapfrog helpers for the kick-drift-kick integrator (y += a * x):
 * y: device double [n]; x: device [n], float when x_is_f32 else double.     */
tp_status tp_axpy(double *y, const void *x, int32_t x_is_f32, double a, int64_t n,
                  void *stream);
/* out = a * x with out float when out_is_f32 else double; x: device double. */
tp_status tp_scale(void *out, int32_t out_is_f32, const double *x, double a, int64_t n,
                   void *stream);

/* Arithmetic peak of this GPU measured by a dependency-free FMA loop:
 * kind 0 = FP32 FFMA, 1 = FP32 packed f32x2 FMA, 2 = FP64 DFMA.  Writes flops
 * per second (an FMA counts 2) to *flops.  Synchronises.                    */
tp_status tp_measure_peak(int32_t kind, double *flops, void *stream);

/* Number of kernels this library launched since it was loaded.             */
int64_t tp_launch_count(void);

/* A static, NUL-terminated English description of s ("unknown status" for a
 * value outside the enum); never NULL, never to be freed; no GPU needed.   */
const char *tp_status_string(tp_status s);

#ifdef __cplusplus
}
#endif
#endif /* TREEPM_SR_H */
