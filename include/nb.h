/*
 * nb.h -- C ABI of the GB300 short-range non-bonded library.
 *
 * The library evaluates short-range non-bonded forces, energies and the virial
 * for a periodic molecular system with the cluster pair algorithm of Pall et
 * al., "Heterogeneous parallelization and acceleration of molecular dynamics
 * simulations in GROMACS" (J. Chem. Phys. 153, 134110 (2020), arXiv:2006.09167):
 *   - atoms are sorted on a grid that is regular in x,y and binned in z into
 *     cells holding a fixed number of atoms; these cells are the 8-atom
 *     clusters, grouped 2x2x2 into super-clusters (Sec. V.A, Fig. 4);
 *   - a bounding-box search builds, per super-cluster, a joint list of
 *     j-clusters with an 8-bit interaction mask telling which of the eight
 *     i-clusters each j-cluster interacts with, plus exclusion bit masks
 *     (Sec. V.A, Sec. V.D);
 *   - an outer list built at a buffered cut-off rlist is pruned by atom-pair
 *     distances into an inner list, in a rolling fashion (Sec. V.D, V.E);
 *   - the pair kernel computes Lennard-Jones plus reaction-field or Ewald
 *     real-space Coulomb interactions over the inner list, each pair once
 *     (Newton's third law), masking excluded pairs and pairs beyond rc (Sec. V.A).
 *
 * Interaction forms (the paper names the interactions but gives no formulas):
 *   V_LJ = C12/r^12 - C6/r^6 - (C12/rc^12 - C6/rc^6)
 *   V_RF = f qi qj (1/r + k_rf r^2 - c_rf), k_rf = (eps_rf-eps_r)/((2 eps_rf+eps_r) rc^3),
 *          c_rf = 1/rc + k_rf rc^2 (eps_rf = +inf: k_rf = 1/(2 rc^3))
 *   V_Ew = f qi qj (erfc(beta r)/r - erfc(beta rc)/rc)
 *   f = 138.935458/eps_r kJ mol^-1 nm e^-2; excluded pairs contribute nothing.
 *   Virial W = -1/2 sum_pairs r_ij (x) F_ij.
 * Units: nm, kJ/mol, e.  Boxes are rectangular; rc < L/2 and rlist < L per axis.
 *
 * Conventions for every call below:
 *   - Pointers named *_dev are device pointers owned by the caller (contiguous,
 *     on the current device).  Pointers named *_host are host pointers.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     Work is enqueued asynchronously on it unless the entry says it synchronises.
 *   - Argument errors found on the host are returned directly and nothing is
 *     enqueued.  Errors found on the device (non-finite coordinates, capacity
 *     overflow) are recorded in a per-context flag read by nb_get_error().
 *   - The context allocates device memory only in nb_create, nb_grid_sort and
 *     nb_pairlist_build.  nb_prune_rolling, nb_forces, nb_forces_vjp and
 *     nb_forces_batched never allocate.
 *   - A context is not thread-safe; calls on one context must be ordered.
 */
#ifndef NB_H
#define NB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct nb_ctx nb_ctx;
typedef struct nb_batch nb_batch;
typedef struct nb_pme nb_pme;

typedef enum {
    NB_OK = 0,
    NB_ERR_INVALID_ARG = 1,   /* bad pointer, size, flag or parameter */
    NB_ERR_BOX_TOO_SMALL = 2, /* rc >= L/2 or rlist >= L on some axis */
    NB_ERR_NOT_READY = 3,     /* call out of order (e.g. forces before a pair list) */
    NB_ERR_CAPACITY = 4,      /* an internal capacity was exceeded (see nb_get_error) */
    NB_ERR_CUDA = 5,          /* a CUDA runtime call failed */
    NB_ERR_TIMEOUT = 6,       /* a bounded device-side wait gave up */
    NB_ERR_NONFINITE = 7      /* non-finite coordinates were seen on the device */
} nb_status;

enum { NB_COULOMB_RF = 0, NB_COULOMB_EWALD = 1, NB_COULOMB_NONE = 2 /* Lennard-Jones only */ };

/* flags of nb_forces / nb_forces_batched */
enum { NB_ENERGY = 1u, NB_VIRIAL = 2u };

/* which list nb_debug_export_pairs exports */
enum { NB_LIST_OUTER = 0, NB_LIST_INNER = 1 };

typedef struct {
    int32_t n_atoms;  /* N >= 1 */
    int32_t n_types;  /* T in [1, 64] */
    int32_t coulomb;  /* NB_COULOMB_RF, NB_COULOMB_EWALD or NB_COULOMB_NONE */
    int32_t reserved; /* must be 0 */
    double eps_r;     /* relative permittivity (> 0) */
    double eps_rf;    /* reaction-field dielectric; +inf (or <= 0) = conducting */
    double beta;      /* Ewald splitting parameter (nm^-1), 0 < beta*rc <= 4 */
    double rc;        /* interaction cut-off (nm) */
    double rlist;     /* outer pair-list cut-off, rlist >= r_in >= rc */
    double r_in;      /* inner (pruned) list cut-off used by nb_pairlist_build */
    const float *c6_host;  /* [T*T] row-major, symmetric, C6 (kJ mol^-1 nm^6) */
    const float *c12_host; /* [T*T] row-major, symmetric, C12 (kJ mol^-1 nm^12) */
} nb_params;

/* Statistics of the current lists (nb_get_stats). */
typedef struct {
    int64_t n_atoms, n_slots, n_clusters, n_superclusters;
    int64_t n_items;        /* work items (super-cluster, shift, j-range chunk) */
    int64_t n_outer_j;      /* j-cluster entries in the outer list */
    int64_t n_outer_bits;   /* set interaction-mask bits in the outer list */
    int64_t n_mask_groups;  /* j-entries carrying explicit exclusion masks */
    int64_t grid_nx, grid_ny;
    int64_t n_launches;     /* kernels this context has launched so far */
} nb_stats;

/* kernels timed by the tracer (nb_trace_read) */
enum { NB_TRACE_FORCES = 0, NB_TRACE_PRUNE = 1, NB_TRACE_GATHER = 2, NB_TRACE_VJP = 3, NB_TRACE_KINDS = 4 };
#define NB_TRACE_ALL ((1 << NB_TRACE_KINDS) - 1) /* nb_trace_enable: every kind */

/* Create a context for one system (Sec. V.A: positions, box, types, charges,
 * exclusions and cut-offs define the problem).  q_host [N] charges, type_host
 * [N] in [0,T), excl_off_host [N+1] / excl_idx_host [excl_off[N]]: symmetric
 * exclusion lists in CSR form (an atom's own index is implicit and must not be
 * listed; at most 16 partners per atom).  All inputs are copied; the caller
 * keeps ownership.  Allocates device memory.  Returns NB_ERR_INVALID_ARG for
 * bad parameters (checked before any CUDA call). */
nb_status nb_create(const nb_params *params, const float *q_host, const int32_t *type_host,
                    const int32_t *excl_off_host, const int32_t *excl_idx_host, nb_ctx **out);

/* Release every resource of the context (NULL is accepted). */
void nb_destroy(nb_ctx *ctx);

/* Replace the charges with q_dev [N] (caller order, device).  Asynchronous. */
nb_status nb_set_charges(nb_ctx *ctx, const float *q_dev, void *stream);

/* Replace the Lennard-Jones tables with c6_dev / c12_dev [T*T] (device,
 * row-major; the pair parameter is (C[a][b] + C[b][a]) / 2).  Asynchronous. */
nb_status nb_set_lj(nb_ctx *ctx, const float *c6_dev, const float *c12_dev, void *stream);

/* Grid sort (Sec. V.A, Fig. 4): bin atoms into xy columns, sort each column
 * by z, cut it into super-cells of 64 atoms, split each super-cell 2x2x2 into
 * 8-atom clusters (z halves, then y halves, then x halves), pad partial
 * clusters, and compute cluster and super-cluster bounding boxes (Sec. V.D).
 * x_dev [N*3] caller-order positions (any periodic image); box_host [3]
 * rectangular box edges.  Each atom's periodic image offset is fixed here and
 * reused until the next grid sort.  Allocates on first use or growth.
 * Invalidates the pair lists. */
nb_status nb_grid_sort(nb_ctx *ctx, const float *x_dev, const double *box_host, void *stream);

/* Bounding-box cluster pair search (Sec. V.A, V.D): for every super-cluster
 * and periodic shift, the joint list of j-clusters whose bounding box lies
 * within rlist of any of its 8 i-cluster boxes, with the 8-bit interaction
 * mask and exclusion bit masks; each cluster pair is listed once (Newton's
 * third law).  Lists are split into chunks and ordered longest first (Sec. V.F).
 * Then prunes the whole list at params.r_in into the inner list (first use,
 * Sec. V.D).  Synchronises `stream` (list sizes are read back to size buffers
 * and launches).  rlist must satisfy params.r_in <= rlist < L. */
nb_status nb_pairlist_build(nb_ctx *ctx, float rlist, void *stream);

/* Rolling prune (Sec. V.E): re-prune part `part` of `n_parts` interleaved
 * parts of the outer list against r_in (rc <= r_in <= rlist), using the
 * positions of the last nb_forces (or nb_grid_sort) call.  For each i-cluster
 * and each half (atoms 0-3, 4-7) of the j-cluster it keeps a bit iff some atom
 * pair of that 8x4 block is closer than r_in (j-cluster splitting); entries
 * with no bit left are dropped.  The outer list is unchanged.  Asynchronous;
 * never allocates. */
nb_status nb_prune_rolling(nb_ctx *ctx, float r_in, int part, int n_parts, void *stream);

/* Forces (Sec. V.A): gathers x_dev [N*3] (caller order) into the cluster
 * layout using the image offsets of the last grid sort, evaluates the inner
 * list and writes f_dev [N*3] (caller order, overwritten).  flags: NB_ENERGY
 * writes e_dev[2] = {E_LJ, E_Coulomb} (FP64, overwritten); NB_VIRIAL writes
 * vir_dev[9] (FP64 row-major, overwritten).  Pair arithmetic and force
 * accumulation are FP32; energies and virial are reduced in FP64.
 * Asynchronous; never allocates; may be captured in a CUDA graph.  Calls on
 * one context (forces, prune, adjoint) must not overlap on the GPU: they share
 * the context's layout, accumulators and work-item counter.  The type-pair
 * tables live in shared memory; beyond about 40 types they exceed 48 KB and the
 * kernel runs at lower occupancy. */
nb_status nb_forces(nb_ctx *ctx, unsigned flags, const float *x_dev, float *f_dev, double *e_dev,
                    double *vir_dev, void *stream);

/* Sorted-layout mode (not in the paper): between two list builds a caller may
 * keep positions and forces in the context's cluster order -- the order the
 * grid sort gives, 64 slots per super-cluster with padding slots -- and so skip
 * the per-step gather of caller-order positions into that order and the scatter
 * of the forces back.  n_slots is nb_stats.n_slots after nb_grid_sort.
 *
 * nb_sorted_export copies to caller buffers the sorted positions and charges of
 * the last grid sort, xq_dev [n_slots*4] (x, y, z, q per slot; positions are the
 * periodic images the sort chose; padding slots hold far-away positions and
 * q = 0), and the permutation perm_dev [n_slots] (caller index of the atom in
 * each slot, -1 for padding; either pointer may be NULL).  Asynchronous.
 * NB_ERR_NOT_READY before the first grid sort. */
nb_status nb_sorted_export(nb_ctx *ctx, float *xq_dev, int32_t *perm_dev, void *stream);

/* Forces at sorted positions xq_dev [n_slots*4] (as exported, x, y, z then moved
 * by the caller; q and the padding slots left as exported).  Writes f_dev
 * [n_slots*4] (force x, y, z per slot, w = 0; padding slots 0; overwritten) and,
 * with NB_ENERGY / NB_VIRIAL, e_dev[2] / vir_dev[9] as nb_forces.  Positions are
 * used as given: no wrapping, no image offsets.  The context keeps xq_dev as the
 * positions of its last force call, which nb_prune_rolling and nb_count_pairs
 * read: it must stay valid and unchanged until they have run (a later nb_forces
 * or nb_grid_sort makes the context use its own copy again).  Asynchronous;
 * never allocates; calls on one context must not overlap on the GPU. */
nb_status nb_forces_sorted(nb_ctx *ctx, unsigned flags, const float *xq_dev, float *f_dev, double *e_dev,
                           double *vir_dev, void *stream);

/* Adjoint of nb_forces (not in the paper): for L = <gF, F> + gE*(E_LJ + E_C),
 * recomputes every pair of the inner list at x_dev and writes gx_dev [N*3],
 * gq_dev [N] (FP32, overwritten) and gc6_dev / gc12_dev [T*T] (FP64,
 * overwritten).  A type pair a != b puts half of its parameter gradient in
 * [a][b] and half in [b][a].  Supports up to 16 atom types (the parameter
 * gradients are accumulated in shared memory); more types return
 * NB_ERR_INVALID_ARG.  Asynchronous; never allocates. */
nb_status nb_forces_vjp(nb_ctx *ctx, const float *x_dev, const float *gF_dev, double gE,
                        float *gx_dev, float *gq_dev, double *gc6_dev, double *gc12_dev,
                        void *stream);

/* nb_forces_vjp with the energy weight read from device memory, gE_dev [1]
 * (FP64), by the adjoint kernel itself: a caller whose gE is the output of an
 * earlier kernel (an autograd backward pass) needs no host synchronisation to
 * read it.  Same outputs and errors as nb_forces_vjp; gE_dev must stay valid
 * until the call's work has run.  Asynchronous; never allocates. */
nb_status nb_forces_vjp_dev(nb_ctx *ctx, const float *x_dev, const float *gF_dev, const double *gE_dev,
                            float *gx_dev, float *gq_dev, double *gc6_dev, double *gc12_dev, void *stream);

/* Batched evaluation of independent systems in one persistent launch
 * (Sec. VI ensembles sharing a GPU; tail balancing of Sec. V.F).  The batch
 * refers to (does not own) `n` contexts that already have pair lists and the
 * same Coulomb type; it must be re-created after any of them is re-built.
 * A pending fused first-use prune (nb_set_fused_prune) is completed here.
 * Allocates in nb_batch_create only. */
nb_status nb_batch_create(nb_ctx *const *ctxs, int n, nb_batch **out);
void nb_batch_destroy(nb_batch *batch);

/* x_dev: concatenated caller-order positions of all systems (system r starts
 * at atom offset sum_{s<r} N_s); f_dev likewise (overwritten); e_dev [n*2],
 * vir_dev [n*9] per system.  Work items of all systems are drawn from one
 * device queue by a persistent kernel.  Asynchronous; never allocates. */
nb_status nb_forces_batched(nb_batch *batch, unsigned flags, const float *x_dev, float *f_dev,
                            double *e_dev, double *vir_dev, void *stream);

/* Counts over the inner (NB_LIST_INNER) or outer (NB_LIST_OUTER) list at the
 * current positions: pairs inside rc that the force kernel computes from it
 * (effective interactions) and atom pairs evaluated (the raw work: 8x8 per
 * mask bit of an outer entry, 8x4 per half-mask bit of an inner entry).  Pairs inside rc that the outer list has and the inner list lacks
 * were missed by the prune.  Synchronises `stream`. */
nb_status nb_count_pairs(nb_ctx *ctx, int which, int64_t *n_within_rc, int64_t *n_evaluated, void *stream);

/* Export the atom pairs the kernel would evaluate from the outer or inner list
 * (mask bit set, both atoms real) as int64 rows (i, j, sx, sy, sz) with
 * pair vector x_i - x_j + s*L in caller coordinates.  Writes at most cap rows
 * to buf_host and the total to *n_total.  For tests; synchronises; allocates
 * temporary device memory. */
nb_status nb_debug_export_pairs(nb_ctx *ctx, int which, int64_t *buf_host, size_t cap,
                                size_t *n_total, void *stream);

/* Copy the sorted layout: perm_host [n_slots] (slot -> caller atom, -1 = pad)
 * and, when not NULL, xq_host [n_slots*4] (x,y,z,q per slot) and
 * bbox_host [n_clusters*8] (lo x,y,z,-, hi x,y,z,-).  For tests; synchronises. */
nb_status nb_debug_layout(nb_ctx *ctx, int32_t *perm_host, float *xq_host, float *bbox_host,
                          void *stream);

nb_status nb_get_stats(nb_ctx *ctx, nb_stats *out);

/* First-use prune fused into the force kernel (Sec. V.D), off by default.  When
 * on, nb_pairlist_build does not prune; the next nb_forces evaluates the outer
 * list, records on the way which (i-cluster, j-half) blocks have an atom pair
 * closer than r_in at that call's positions, and compacts them into the inner
 * list (the same list the separate prune gives at those positions).  Calls that
 * need the inner list before that force call (nb_prune_rolling, nb_forces_vjp,
 * nb_forces_batched, inner-list counts and exports) prune it first.  Takes effect
 * at the next nb_pairlist_build.  on: 0 or 1. */
nb_status nb_set_fused_prune(nb_ctx *ctx, int on);

/* Tuning (Sec. V.F: lists are split when there are too few of them for the GPU):
 * the largest number of outer j-cluster entries per work item (4..128, default
 * 16).  Takes effect at the next nb_pairlist_build. */
nb_status nb_set_split(nb_ctx *ctx, int max_entries_per_item);

/* Tuning (not in the paper): the number of column segments of the pair search,
 * 1..8, or 0 (the default) for the library's choice.  Each super-cluster's
 * j-list is searched by that many warps, warp g taking the grid columns with
 * index = g (mod segments), and each work item then holds the entries of one
 * shift and one segment.  The library's choice doubles the segments from 1 while
 * the search would have fewer than 12,000 warps (8 for a 96k-atom water box, 1
 * for 1.5M atoms).  The pair set is the same for every value; the item structure,
 * and with it the work balance of the force kernels, is not.  Takes effect at the
 * next nb_pairlist_build; NB_ERR_INVALID_ARG outside 0..8. */
nb_status nb_set_search_segments(nb_ctx *ctx, int segments);

/* Tracing (not in the paper): CUDA events are recorded on the launch stream
 * around every kernel of the kinds selected by `kinds` (bit NB_TRACE_x set:
 * kind x is traced; 0 turns tracing off; other bits: NB_ERR_INVALID_ARG) of
 * this context, at most 65536 launches per kind between reads.  Each traced
 * launch adds two event records to its stream, so a caller may trace a sample
 * of launches by switching the selection between calls: launches traced so far
 * stay pending until nb_trace_read returns them.  The first enabling creates
 * the events (host resources); not allowed during stream capture. */
nb_status nb_trace_enable(nb_ctx *ctx, int kinds);

/* Device time of the traced launches of one kind since the last read:
 * *total_ms (sum of event intervals) and *n_launches.  Synchronises on the
 * recorded events and resets the counters of that kind. */
nb_status nb_trace_read(nb_ctx *ctx, int kind, double *total_ms, int64_t *n_launches);

/* Return (and clear) the first device-side error recorded since the last
 * call; synchronises `stream`. */
nb_status nb_get_error(nb_ctx *ctx, void *stream);

const char *nb_status_str(nb_status s);

/* ------------------------------------------------------------------------
 * Completing the Ewald sum.  The short-range kernel computes the real-space
 * term of non-excluded pairs inside rc (Sec. V.A); the paper runs the
 * reciprocal part as a separate PME task on its own stream (Sec. IV).  With the
 * self and exclusion terms below the four parts give the Ewald sum of a neutral
 * periodic system with tin-foil boundaries:
 *   E = E_real + E_recip + E_self + E_excl,  E_self = -f beta/sqrt(pi) sum q^2,
 *   E_excl = -f sum_{excluded pairs} qi qj erf(beta r)/r,  f = 138.935458/eps_r.
 * Virials use the convention of nb_forces (W = -1/2 sum r (x) F). */

/* Smooth PME (cardinal B-spline charge assignment of order `order`, 3-D FFT on
 * a K1 x K2 x K3 grid, influence function, inverse FFT, force gather). */
typedef struct {
    int n_atoms;
    int grid[3];   /* K1, K2, K3 (each >= 2*order, <= 4096) */
    int order;     /* B-spline order, 3..8 (4 is the usual choice) */
    int reserved;  /* must be 0 */
    double beta;   /* Ewald splitting parameter (nm^-1), > 0: the short-range part's */
    double eps_r;  /* relative dielectric constant, > 0 */
} nb_pme_params;

/* Allocates the grids and the FFT plans (cuFFT) on the current device. */
nb_status nb_pme_create(const nb_pme_params *params, nb_pme **out);
void nb_pme_destroy(nb_pme *pme);

/* Reciprocal-space energy, forces and virial at positions x_dev [N*3] (caller
 * order, any periodic image) with charges q_dev [N] (device) in the
 * rectangular box box_host [3].  Forces are ADDED to f_dev [N*3] (so that they
 * can follow nb_forces on the same buffer); with NB_ENERGY e_dev[0] = E_recip
 * (FP64, overwritten), with NB_VIRIAL vir_dev[9] (FP64, overwritten).  Weights,
 * grid and FFTs are FP32 (fractional coordinates FP64), energy and virial sums
 * FP64.  Asynchronous on `stream`; never allocates; calls on one nb_pme must
 * not overlap on the GPU. */
nb_status nb_pme_forces(nb_pme *pme, unsigned flags, const float *x_dev, const float *q_dev, const double *box_host,
                        float *f_dev, double *e_dev, double *vir_dev, void *stream);

/* Exclusion and self terms of a context built with NB_COULOMB_EWALD, at
 * positions x_dev [N*3] (caller order), with its charges, exclusions, beta and
 * the box of its last grid sort.  Forces are ADDED to f_dev [N*3]; with
 * NB_ENERGY e_dev[2] = {E_excl, E_self} (overwritten); with NB_VIRIAL
 * vir_dev[9] = W_excl (overwritten).  NB_ERR_INVALID_ARG for other Coulomb
 * types, NB_ERR_NOT_READY before the first grid sort.  Asynchronous; never
 * allocates. */
nb_status nb_ewald_corrections(nb_ctx *ctx, unsigned flags, const float *x_dev, float *f_dev, double *e_dev,
                               double *vir_dev, void *stream);

/* ------------------------------------------------------------------------
 * Allocation-free evaluation of one small system.  The paper has no
 * counterpart: it exists for callers that cannot allocate device memory, such
 * as code whose device memory belongs to another allocator (a framework's
 * caching allocator, or a pool reserved at start-up), code that is not allowed
 * to allocate once it is running, and latency-critical code that cannot risk
 * the device synchronisation cudaMalloc/cudaFree may cause.  It needs no
 * context and no pair list: all pairs of the system are evaluated with the same
 * pair interactions as nb_forces (inputs: params (rlist and r_in are ignored),
 * x_dev [N*3], q_dev [N], type_dev [N] with every type in [0, n_types),
 * optional device exclusion CSR excl_off_dev [N+1] / excl_idx_dev (both NULL
 * for none, at most 16 partners per atom), box_host [3]; outputs as nb_forces:
 * f_dev [N*3] overwritten, e_dev [2] with NB_ENERGY, vir_dev [9] with
 * NB_VIRIAL).
 *
 * Its scratch is a file-scope static device array of about 410 KB that every
 * GPU loading the library holds until the process exits.  Limits: N <=
 * NB_NOALLOC_MAX_ATOMS and T <= NB_NOALLOC_MAX_TYPES; larger sizes return
 * NB_ERR_CAPACITY before any work is enqueued.  Types and exclusion rows live
 * in device memory, so they are checked on the device: if any type lies
 * outside [0, T) or any exclusion row is malformed or longer than 16 entries,
 * the call still returns NB_OK but writes NaN to every force component and to
 * every requested energy and virial entry.  The first call on a device looks
 * up the array's device address (cudaGetSymbolAddress) with that device current
 * and keeps it for the life of the process; make that first call before any
 * stream capture, and do not use this entry point on a device after
 * cudaDeviceReset (the address it kept is then stale).  All calls share the one
 * array (each call clears its status word and overwrites what it reads), so
 * calls whose work overlaps on the GPU -- e.g. on two streams without ordering
 * -- race and give wrong results; order them on one stream.  Never allocates.
 * Intended for small systems: the work is O(N^2). */
#define NB_NOALLOC_MAX_ATOMS 16384
#define NB_NOALLOC_MAX_TYPES 8
nb_status nb_forces_small_noalloc(const nb_params *params, const float *x_dev, const float *q_dev,
                                  const int32_t *type_dev, const int32_t *excl_off_dev,
                                  const int32_t *excl_idx_dev, const double *box_host, unsigned flags,
                                  float *f_dev, double *e_dev, double *vir_dev, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* NB_H */
