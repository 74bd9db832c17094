/*
 * otoo.h -- C ABI of the GB300 octree force library.
 *
 * The library splits one softened-gravity force step the way the paper's
 * heterogeneous code does (Section I and the step list of Section V: the CPU
 * builds the tree and the cell properties, the GPU evaluates the forces):
 *
 *   host   otoo_build_tree            octree over one particle system
 *          otoo_make_groups_and_lists groups of up to n_crit particles and one
 *                                     shared interaction list per group
 *          otoo_pack_batch            several systems in one ragged buffer
 *          otoo_make_plan             load-balanced work items for the device
 *   device otoo_force                 acceleration and potential of every group
 *                                     particle against every entry of its list
 *          otoo_force_host            the same from host buffers (copies inside)
 *          otoo_mlp_*                 learned opening-angle network (forward,
 *                                     backward, Adam step, theta choice)
 *
 * Conventions
 *  - Every function returns 0 on success or a negative OTOO_E* code; the
 *    message of the last error on the calling thread is otoo_last_error().
 *    No C++ exception crosses this boundary.
 *  - Host handles (otoo_tree, otoo_lists, otoo_plan) are owned by the library
 *    and released with their *_free function.  Pointers returned by the
 *    *_export functions stay valid until that handle is freed.
 *  - Device buffers are owned by the caller.  Device functions are
 *    asynchronous on the given stream (a cudaStream_t passed as void*; NULL is
 *    the legacy default stream).  Errors detected by a kernel are written to
 *    the caller's status word and read by otoo_check_status after a sync.
 *  - Positions are FP64, masses FP32, G = 1.  Outputs are FP64.
 *  - Particle ("tree") order: the host library sorts particles along a Hilbert
 *    curve.  perm[k] is the caller's index of tree particle k; otoo_force writes
 *    its outputs at perm[k] when a perm array is supplied.
 */
#ifndef OTOO_H
#define OTOO_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes ---------------------------------------------------------- */
#define OTOO_OK       0
#define OTOO_EINVAL  -1   /* bad argument: size, pointer, non-finite input, eps <= 0 */
#define OTOO_ENOMEM  -2   /* host allocation failed */
#define OTOO_ECUDA   -3   /* a CUDA runtime call failed */
#define OTOO_EDEVICE -4   /* a kernel reported bad data (status word) */

/* precision of otoo_force */
#define OTOO_FP32K 0      /* FP32 centre-relative pairs, per-thread Kahan sums, FP64 final sums */
#define OTOO_FP64  1      /* every pair in FP64 (comparison form) */

/* ---- parameters ----------------------------------------------------------- */
/* acceptance rule of the walk (otoo_params.mac) */
#define OTOO_MAC_THETA 0  /* opening angle theta (group MAC of Barnes 1990, Section III-D) */
#define OTOO_MAC_SW    1  /* Salmon-Warren absolute MAC, Section II-B Eq. SW_MAC */
#define OTOO_MAC_SPH   2  /* SPH neighbours (Section II, Eq. SPH_RAD): lists of particles only */

typedef struct otoo_params {
    double theta;                  /* opening angle; 0 = open every cell (direct sum) */
    int32_t leaf_size;             /* max particles per tree leaf (>= 1) */
    int32_t n_crit;                /* max particles per group (>= 1, <= 1024) */
    int32_t use_quad;              /* 1 = cells carry a quadrupole */
    int32_t mac;                   /* OTOO_MAC_THETA, OTOO_MAC_SW or OTOO_MAC_SPH */
    double eps;                    /* Plummer softening length (> 0) */
    const float* theta_per_group;  /* host, NULL = fixed theta; else one angle per group
                                      in the group order of a previous call on the
                                      same tree with the same n_crit (OTOO_MAC_THETA only) */
    double delta;                  /* OTOO_MAC_SW: accuracy parameter (an acceleration,
                                      G = 1); 0 = accept no cell */
    double m_limit;                /* OTOO_MAC_SW: cells heavier than this are never
                                      accepted (Section III-C); <= 0 = no limit */
    const float* h_sph;            /* OTOO_MAC_SPH: host, one neighbour radius h > 0 per
                                      particle, caller order */
} otoo_params;

typedef struct otoo_tune {
    int32_t block;                 /* threads per CTA: 64, 128 or 256 (the FP32 form runs
                                      one independent work item per warp; block, iblock
                                      and tile must name a compiled variant) */
    int32_t iblock;                /* target particles per thread: 1, 2 or 4; a work item
                                      holds at most 32 * iblock targets */
    int32_t tile;                  /* list entries per staged tile: 64, 128 or 256 (FP32
                                      form; the FP64 form stages 128 entries per tile) */
    int32_t split;                 /* max list entries per work item (>= 32) */
    int32_t ctas_per_sm;           /* resident CTAs per SM for the persistent grid (0 = auto) */
    int32_t packed;                /* FP32 form: 1 = pairs of list entries evaluated with packed
                                      two-wide FP32 instructions, 0 = one entry at a time */
} otoo_tune;

/* ---- device-side layout (what the host library exports and the caller
        uploads; every array is 16-byte aligned and tightly packed, quad and the
        split scratch 32-byte aligned) ----------------------------------------- */

/* A source: a particle (index < n_part) or a cell (index >= n_part).  For a
   cell, (x, y, z) is its centre of mass and m its mass. 32 bytes. */
typedef struct otoo_src {
    double x, y, z;
    float m;
    int32_t pad;
} otoo_src;

/* Quadrupole of cell (n_part + k), k in [0, n_cell): the traceless
   Q_ab = sum m (3 d_a d_b - |d|^2 delta_ab), d = x - com, and b2 = B_2 =
   sum m |d|^2 (Eq. B2; the trace of the second moment), which the softened
   quadrupole term needs: with q = (r^2 + eps^2)^(-1/2) and w = r.Q.r -
   b2 eps^2, a cell adds -(1/2) w q^5 to the potential and
   (5/2) w q^7 r - q^5 Q r to the acceleration (r = com - x), the
   second-order Taylor term of the softened pair law.  32 bytes. */
typedef struct otoo_quad {
    float xx, yy, zz, xy, xz, yz, b2, pad;
} otoo_quad;

/* One group: particles [first, first + count) in tree order share the list
   entries [list_off, list_off + n_cell + n_part): n_cell cell indices first,
   then n_part particle indices.  64 bytes. */
typedef struct otoo_group {
    int32_t first, count, n_cell, n_part;
    int64_t list_off;
    double eps2;                   /* softening^2 of the group's system */
    double cx, cy, cz;             /* FP64 group centre (centre of the particles' box) */
    float theta;                   /* opening angle the list was made with */
    int32_t sys;                   /* system index within a batch */
} otoo_group;

/* One work item: target particles [i0, i0 + ni) of group g (relative to the
   group's first particle) against list entries [j0, j1) (relative to the
   group's list).  slot < 0: the item covers the whole list and writes the
   outputs; slot >= 0: the item writes FP64 partial sums at
   partial[(slot * n_crit_max + i) * 4 + 0..3] and otoo_force merges the list
   chunks of each group in chunk order.  32 bytes. */
typedef struct otoo_item {
    int32_t g, i0, ni, j0, j1, slot, pad0, pad1;
} otoo_item;

/* A group whose list was split: its chunks' partials start at slot0 and run
   over n_chunks consecutive slots. 16 bytes. */
typedef struct otoo_split {
    int32_t g, slot0, n_chunks, pad;
} otoo_split;

/* Device view of one step's inputs (all pointers device, caller-owned). */
typedef struct otoo_dev_system {
    int64_t n_part;                /* target particles (tree order) */
    int64_t n_src;                 /* n_part + number of cells */
    int64_t n_list;                /* entries in list */
    int64_t partial_doubles;       /* length of partial in doubles; a work item or split whose
                                      slots reach past it is skipped and flagged (OTOO_EDEVICE) */
    int32_t n_groups, n_items, n_splits, n_crit_max;
    const otoo_src* src;           /* [n_src] */
    const otoo_quad* quad;         /* [n_src - n_part], NULL = monopole cells; 32-byte aligned */
    const otoo_group* groups;      /* [n_groups] */
    const int32_t* list;           /* CSR source indices */
    const otoo_item* items;        /* [n_items], in launch order */
    const otoo_split* splits;      /* [n_splits] */
    const int64_t* perm;           /* [n_part] output index of each tree particle, NULL = tree order */
    double* partial;               /* scratch, partial_doubles doubles (>= the plan's
                                      otoo_plan_info.partial_doubles) */
    uint32_t* counter;             /* scratch, >= 4 uint32 (work ticket and status) */
    void* split;                   /* scratch for OTOO_FP32K, >= 32 * n_src bytes, 32-byte aligned: each source's
                                      position as a float pair (hi = x rounded to FP32,
                                      lo = x - hi rounded) and its mass */
} otoo_dev_system;

/* ---- opaque host handles ------------------------------------------------- */
typedef struct otoo_tree otoo_tree;
typedef struct otoo_lists otoo_lists;
typedef struct otoo_plan otoo_plan;

/* Host arrays of a lists object (pointers owned by the lists handle). */
typedef struct otoo_lists_view {
    int64_t n_part, n_src, n_groups, n_list;
    int32_t n_sys, use_quad;
    const otoo_src* src;           /* [n_src] */
    const otoo_quad* quad;         /* [n_src - n_part] (zeros when use_quad = 0) */
    const otoo_group* groups;      /* [n_groups] */
    const int32_t* list;           /* [n_list] */
    const int64_t* perm;           /* [n_part] caller index of each tree particle */
    const int64_t* sys_part_off;   /* [n_sys + 1] first tree particle of each system */
    int64_t interactions;          /* sum over groups of count * (n_cell + n_part) */
    int64_t cell_interactions;     /* part of it with cell entries */
} otoo_lists_view;

typedef struct otoo_plan_info {
    int64_t n_items, n_splits;
    int64_t partial_doubles;       /* scratch size otoo_force needs */
    int32_t n_crit_max;
    int32_t pad;
    const otoo_item* items;        /* host [n_items] */
    const otoo_split* splits;      /* host [n_splits] */
} otoo_plan_info;

/* ---- host library ------------------------------------------------------------ */

/* Build the octree of n particles (Section III-B: root cube, keys, sort,
   linked cells; Section III-C: cell mass, centre of mass; the quadrupole is
   this library's extension).  pos: host [n][3] FP64 row-major; mass: host [n]
   FP32, > 0.  Root cube: centred on the bounding box, side = max extent *
   (1 + 1e-12); particles are quantised to a 2^21 grid per axis and sorted by
   (Hilbert key, index).  Copies its inputs.  Errors: OTOO_EINVAL for n < 1,
   NULL pointers, non-finite positions or masses <= 0; OTOO_ENOMEM. */
int otoo_build_tree(const double* pos, const float* mass, int64_t n,
                    const otoo_params* params, otoo_tree** out);

/* Groups and lists (Section III-D, the vectorised walk of Barnes 1990 done on
   the host): groups are the maximal cells with at most n_crit particles; each
   group walks the tree once.  With OTOO_MAC_THETA it accepts cell c when c's
   cube does not overlap the group's box and d_min > l_c / theta + s_c (d_min:
   distance from c's centre of mass to the box, l_c: cube side, s_c: distance
   from the centre of mass to the cube centre); params->theta_per_group, when
   set, overrides theta group by group.  With OTOO_MAC_SW it accepts c when
   d_min > r_b = b_max / 2 + sqrt(b_max^2 / 4 + sqrt(3 B_2 / delta)) (Eq.
   SW_MAC; B_2 = sum m |x - com|^2, Eq. B2; b_max = max |x - com|), with r_b
   = 2 S_root for cells heavier than m_limit (S_root: root cube side), and
   the group records carry theta = 0.  With OTOO_MAC_SPH a cell whose
   r_SPH = max_j (|x_j - com| + h_j) (Eq. SPH_RAD) is smaller than d_min is
   skipped (it holds no neighbour of any group particle) instead of entered,
   so the lists hold particles only (n_cell = 0).  Rejected leaves contribute
   their particles.  Errors: OTOO_EINVAL (eps <= 0, n_crit < 1 or > 1024, theta < 0,
   unknown mac, delta < 0 or not finite), OTOO_ENOMEM. */
int otoo_make_groups_and_lists(const otoo_tree* tree, const otoo_params* params,
                               otoo_lists** out);

/* Concatenate the lists of n_sys systems into one ragged buffer: particles of
   all systems first (system by system), then all cells; group and list
   indices are rebased.  The inputs stay owned by the caller. */
int otoo_pack_batch(const otoo_lists* const* per_sys, int32_t n_sys, otoo_lists** out);

/* Work items for otoo_force: every group is cut into particle chunks of at
   most 32 * tune->iblock particles whose sizes fill a warp's lanes (a fixed
   table per iblock, the cut of each group size that minimises a modelled
   warp time: pair steps of ceil(ni / iblock) lanes in 32 / that many lane
   subsets, staging of the list once per chunk, a fixed cost per item, the
   subset merge; e.g. 26 particles at iblock 2 become chunks of 10 and 16),
   lists longer than tune->split entries into chunks of at most tune->split
   entries (of balanced length); items are ordered by decreasing cost ni *
   (j1 - j0) (longest processing time first).  Groups with an empty list (a
   negative per-group angle) get no item.  The device plan (otoo_plan_count,
   otoo_plan_fill) makes the same items.  Errors: OTOO_EINVAL (a group of
   more than 1024 particles), OTOO_ENOMEM. */
int otoo_make_plan(const otoo_lists* lists, const otoo_tune* tune, otoo_plan** out);

/* Host arrays of a tree (pointers owned by the tree handle); cells are
   numbered from 0 (the root), cell k is source n_part + k, the children of a
   cell are consecutive. */
typedef struct otoo_tree_view {
    int64_t n_part, n_cell;
    int32_t depth, leaf_size;
    double root_lo[3], root_side;
    const double* pos;             /* [n_part][3] tree order */
    const float* mass;             /* [n_part] tree order */
    const int64_t* perm;           /* [n_part] caller index of each tree particle */
    const int64_t* cell_begin;     /* [n_cell] first tree particle */
    const int64_t* cell_end;       /* [n_cell] one past the last */
    const int32_t* cell_level;     /* [n_cell] 0 = root */
    const int32_t* cell_nchild;    /* [n_cell] 0 = leaf */
    const int64_t* cell_child0;    /* [n_cell] first child cell */
    const int64_t* cell_org;       /* [n_cell][3] integer origin on the 2^21 grid */
    const double* cell_com;        /* [n_cell][3] */
    const double* cell_mass;       /* [n_cell] */
    const double* cell_quad;       /* [n_cell][6] Qxx Qyy Qzz Qxy Qxz Qyz */
    const double* cell_b2;         /* [n_cell] B_2 = sum m |x - com|^2 (Eq. B2) */
    const double* cell_bmax;       /* [n_cell] b_max = max |x - com| */
} otoo_tree_view;

int otoo_tree_export(const otoo_tree* tree, otoo_tree_view* view);
int otoo_lists_export(const otoo_lists* lists, otoo_lists_view* view);
int otoo_plan_export(const otoo_plan* plan, otoo_plan_info* info);

/* Per-group features for the learned opening angle (statistics of each
   group's list): feat[g][0..4] = log2(list length), log10 of the minimum over
   cell entries of d_min / l_c (3.0 when the list has no cell entry),
   log10(box half-diagonal / eps) (box half-diagonal floored at eps / 1000),
   cell mass fraction of the list, and log10 of the list's relative
   truncation estimate sum_cells B_2 b_max / d_c^5 over |a_net| (B_2, b_max:
   the cell's spread, Eq. B2; d_c: distance of its centre of mass to the
   group box; a_net: the softened pull of all entries at the group centre;
   floored at 1e-12).  host out [n_groups][5]. */
int otoo_group_features(const otoo_tree* tree, const otoo_lists* lists, float* feat);

void otoo_tree_free(otoo_tree* tree);
void otoo_lists_free(otoo_lists* lists);
void otoo_plan_free(otoo_plan* plan);

/* ---- device -------------------------------------------------------------------- */

/* Default tuning for a given n_crit. */
int otoo_default_tune(int32_t n_crit, otoo_tune* tune);

/* Softened acceleration and potential (Section II: particle-particle and
   particle-cell interactions, the monopole and this library's quadrupole
   extension; Plummer softening with the group's eps2):
     a_i = sum_j m_j r / (r^2 + eps^2)^(3/2) [+ quadrupole terms],
     phi_i = -sum_j m_j / (r^2 + eps^2)^(1/2) [+ ...],   r = x_j - x_i, j != i.
   sys: device view, all arrays device-resident; accel: [n_part][3] FP64;
   pot: [n_part] FP64; both indexed by perm when sys->perm is set.  accel and
   pot are device memory or pinned (page-locked) host memory, which the GPU
   addresses directly: the kernel then writes the results into host memory
   as it goes, and they are there when the stream has finished (on GB300 the
   host link takes these writes during the kernel, which replaces the copy
   that would follow it).
   precision: OTOO_FP32K or OTOO_FP64.  tune: the tuning the plan was made with.
   The step (ticket reset, persistent force kernel, chunk merge) is recorded
   once per distinct argument set into a CUDA graph and replayed on stream.
   Every work item, list index and split record is bounds-checked on the
   device before it is used (groups, list, sources, and the partial slots
   against sys->partial_doubles); a bad one is skipped, its targets are not
   written, and the status word records it for otoo_check_status.
   Errors: OTOO_EINVAL (sizes, NULL pointers, tune, split lists without
   partial scratch of at least 4 * n_crit_max doubles), OTOO_ECUDA. */
int otoo_force(const otoo_dev_system* sys, double* accel, double* pot, int32_t precision,
               const otoo_tune* tune, void* stream);

/* Same computation from HOST arrays: the library copies the lists view and
   the plan to its own device buffers, runs otoo_force on stream and copies
   accel/pot (host, caller order) back; returns after the stream has synced.
   When accel and pot are both pinned (page-locked) host memory the kernel
   writes them directly and no copy follows it.  Device buffers are kept for
   the next call of the same size. */
int otoo_force_host(const otoo_lists_view* lists, const otoo_plan_info* plan, double* accel,
                    double* pot, int32_t precision, const otoo_tune* tune, void* stream);

/* The centre-relative coordinates the FP32 form computes (the group-centre
   subtraction of its FP32 pairs; the paper's single-precision kernel works
   on absolute coordinates), exposed for checks:
   out[s][a] = ((hi - c_a) + lo) in FP32, where (hi, lo) is the float pair
   of src[s]'s coordinate a (hi = x rounded to FP32, lo = (x - hi) rounded)
   and c_a = c[a] rounded to FP32 -- the same k_split and the same device
   function as the force kernels' staging.  src: device [n]; c: host, 3
   doubles; out: device [n][3] FP32; scratch: device, 32 * n bytes, 32-byte
   aligned.  Asynchronous on stream.  Errors: OTOO_EINVAL, OTOO_ECUDA. */
int otoo_centre_relative(const otoo_src* src, int64_t n, const double* c, float* out, void* scratch, void* stream);

/* Reads the status word a previous otoo_force wrote (device counter[1]);
   returns OTOO_EDEVICE if a kernel flagged bad data.  Synchronises stream. */
int otoo_check_status(const otoo_dev_system* sys, void* stream);

/* The force step of otoo_force for callers that cannot allocate device
   memory: the work ticket, the status word, the per-step float pairs of the
   FP32 form and the chunk partials of split lists live in a device array
   that the library declares at file scope, so the call itself allocates
   nothing (no cudaMalloc or cudaFree, directly or through any library).
   Such callers include code running under a device-memory budget owned by
   someone else (a host application's pool allocator that already holds the
   GPU's memory, an embedding runtime whose allocator must not be bypassed),
   and latency-critical loops that must not enter the CUDA runtime's allocator.
   There is no counterpart in the paper; this is a deployment option.
     sys:       as for otoo_force; its partial, partial_doubles, counter and
                split fields are ignored (the array is used instead).
     partial_doubles: the plan's otoo_plan_info.partial_doubles (the part of
                the array given to the chunk partials; work items whose slots
                reach past it are skipped and flagged, as in otoo_force).
     Scratch limit: otoo_force_static_capacity() bytes (16 MiB), shared as
                256 bytes + 32 * n_src bytes (OTOO_FP32K only) + 8 *
                partial_doubles bytes, each part rounded up to 256 bytes;
                a larger step is rejected with OTOO_EINVAL before any launch.
   Every GPU that loads the library holds the 16 MiB array until the process
   exits.  The first call on a device looks up the array's device address
   (cudaGetSymbolAddress, once per device, with that device current); make
   that first call before any stream capture.  Every call on a device uses
   the same array and leaves its contents behind; the ticket and status word
   are cleared by each call, everything else is overwritten before it is
   read.  Calls whose work overlaps on the GPU (other streams, other host
   threads) race on the array: serialise them.  The kernels are launched
   directly on stream, asynchronously; the call's status word lives in the
   array and is read by otoo_force_static_status.  The array's address is
   cached per device for the life of the process: do not use this call on a
   device after cudaDeviceReset (the module is reloaded at a new address). */
int otoo_force_static(const otoo_dev_system* sys, int64_t partial_doubles, double* accel, double* pot,
                      int32_t precision, const otoo_tune* tune, void* stream);

/* Status of the last otoo_force_static on the current device: copies the
   status word out of the library's array on stream and synchronises it;
   OTOO_EDEVICE when a kernel skipped a bad work item or list index, OTOO_OK
   otherwise (also before any call).  Allocates nothing. */
int otoo_force_static_status(void* stream);

/* Size in bytes of the array otoo_force_static uses. */
int64_t otoo_force_static_capacity(void);

/* FP64 direct sum (Section II: the O(N^2) sum a tree code approximates),
   used as the exact reference of the learned opening angle's training
   errors:  for each target t, i = targets[t] (an index into src),
     accel[t] = sum_{j != i} m_j r / (r^2 + eps2)^(3/2),
     pot[t]   = -sum_{j != i} m_j / (r^2 + eps2)^(1/2),   r = x_j - x_i,
   over the n_src sources src[0, n_src) (pass the particles only).
   Device arrays: src [n_src], targets [n_tgt] int64, accel [n_tgt][3],
   pot [n_tgt], scratch >= 4 * otoo_direct_chunks(n_src, n_tgt) * n_tgt
   doubles, status one uint32 (bit 2 set when a target index is out of
   range).  Asynchronous on stream; deterministic (chunk sums in order). */
int64_t otoo_direct_chunks(int64_t n_src, int64_t n_tgt);
int otoo_direct(const otoo_src* src, int64_t n_src, const int64_t* targets, int64_t n_tgt, double eps2,
                double* accel, double* pot, double* scratch, uint32_t* status, void* stream);

/* Arithmetic throughput probe, the measured counterpart of the peak the FP32
   form's roofline divides by (not part of the force step): a grid of all
   resident 256-thread blocks, each thread running 8 independent chains of
   iters dependent operations of one kind: 0 scalar fma.rn.f32 (2 flop
   each), 1 packed fma.rn.f32x2 (4 flop each), 2 fma.rn.f64 (2 flop each),
   3 rsqrt.approx.ftz.f32 (1 operation each).  *flops (host) receives the
   operation count of the launch (flop for kinds 0-2); time the call with
   CUDA events on stream.  sink: device, otoo_fma_probe_threads() floats
   (never written in practice; it keeps the chains live).  Errors:
   OTOO_EINVAL, OTOO_ECUDA. */
int64_t otoo_fma_probe_threads(void);
int otoo_fma_probe(int32_t iters, int32_t kind, float* sink, double* flops, void* stream);

/* ---- the walk on the device ------------------------------------------------------
   Section III-D: the paper walks the tree on the GPU, one group of particles
   sharing one traversal (Barnes 1990), with the group-to-cell minimum
   distance in the acceptance test.  Here one warp walks one group.  The
   lists are the ones otoo_make_groups_and_lists makes on the host for the
   same tree and parameters: the same cell entries and the same particle
   entries per group (each run -- cells, then particles -- in the walk's own
   order, which may differ from the host's), because every acceptance test
   takes the host's decision: an FP32 filter decides when the FP32 value is
   provably on the same side of the threshold (margin 2^-16 of the squared
   scale of the test; the rounding bound is below 2^-18), otherwise the FP64
   test of the host walk runs, operation for operation.

   Host preparation: otoo_find_groups (group ranges), otoo_tree_device_arrays
   (sources, quadrupoles and walk records); device: otoo_walk_count,
   otoo_walk_fill, then otoo_plan_count / otoo_plan_fill for the work items of
   otoo_force. */

/* Walk record of cell k (64 bytes): the FP32 data of the filter and the
   tree links. */
typedef struct otoo_wcell {
    float com_hi[3];               /* centre of mass rounded to FP32 */
    float com_lo[3];               /* (com - com_hi) rounded to FP32 */
    float e[3];                    /* (com - cube lower corner) rounded, in [0, side] */
    float side;                    /* cube side rounded */
    float s;                       /* |com - cube centre| (FP64, as the host test computes it) rounded */
    int32_t child0, nchild;        /* children [child0, child0 + nchild), nchild = 0 for a leaf */
    int32_t begin, end;            /* tree-order particle range */
    float rb;                      /* OTOO_MAC_SW: bounding radius r_b rounded (infinite when
                                      delta = 0); OTOO_MAC_SPH: r_SPH rounded; 0 for the
                                      opening angle */
} otoo_wcell;

/* FP64 geometry of cell k (96 bytes): what the exact test reads. */
typedef struct otoo_wcell64 {
    double lo[3];                  /* cube lower corner */
    double side;                   /* cube side */
    double com[3];                 /* centre of mass */
    double gc[3];                  /* cube centre */
    double rb;                     /* OTOO_MAC_SW / OTOO_MAC_SPH: r_b or r_SPH as the host walk
                                      computes it; else 0 */
    double pad;
} otoo_wcell64;

/* Groups of otoo_make_groups_and_lists (maximal cells with at most n_crit
   particles, in tree order; a last-level leaf with more particles cut into
   chunks of n_crit): first[g], count[g], host arrays of capacity entries.
   *n_groups receives the number of groups.  first/count may be NULL with
   capacity 0 to query the number.  Errors: OTOO_EINVAL (n_crit outside
   [1, 1024], capacity too small when arrays are given). */
int otoo_find_groups(const otoo_tree* tree, int32_t n_crit, int32_t* first, int32_t* count,
                     int64_t capacity, int64_t* n_groups);

/* Device inputs of the walk and the force step from a tree, into host arrays
   the caller allocated (any may be NULL to skip it): src [n_part + n_cell]
   (particles in tree order, then cells: centre of mass, mass) and quad
   [n_cell] exactly as otoo_make_groups_and_lists stores them (zeros when
   use_quad = 0); cell [n_cell] and cell64 [n_cell] walk records.  params
   (may be NULL: opening angle) selects the acceptance rule the records are
   for; with OTOO_MAC_SW the records carry r_b for params->delta and
   params->m_limit, with OTOO_MAC_SPH r_SPH for params->h_sph. */
int otoo_tree_device_arrays(const otoo_tree* tree, int32_t use_quad, const otoo_params* params, otoo_src* src,
                            otoo_quad* quad, otoo_wcell* cell, otoo_wcell64* cell64);

/* Device view of one walk (all pointers device, caller-owned). */
typedef struct otoo_dev_walk {
    int64_t n_part, n_cell;        /* the tree's particles and cells */
    int32_t n_groups;
    int32_t exact;                 /* 1 = every acceptance test in FP64 (no FP32 filter) */
    int32_t mac;                   /* OTOO_MAC_THETA, OTOO_MAC_SW or OTOO_MAC_SPH (records made
                                      for it; OTOO_MAC_SPH enters no cell) */
    int32_t set;                   /* groups one warp walks together (consecutive in group
                                      order; each cell's record loaded once and tested per
                                      group): 1..8, or 0 = up to 8 while every resident warp
                                      gets about three sets.  Same entries per group for
                                      every value (their order within a group may differ).
                                      Other values: OTOO_EINVAL */
    double theta;                  /* opening angle when theta_per_group is NULL (>= 0) */
    double eps2;                   /* softening^2, copied into every group record */
    const otoo_src* src;           /* [n_part + n_cell]: particle positions (tree order) */
    const otoo_wcell* cell;        /* [n_cell] */
    const otoo_wcell64* cell64;    /* [n_cell] */
    const int32_t* group_first;    /* [n_groups] */
    const int32_t* group_count;    /* [n_groups], each in [1, 1024] */
    const float* theta_per_group;  /* [n_groups] or NULL; a negative angle skips the group */
    uint32_t* counter;             /* scratch, >= 4 uint32: work ticket, status */
    int64_t* totals;               /* >= otoo_walk_totals_len(n_groups) int64: [0] list
                                      entries, [1] interactions, [2] cell interactions,
                                      [3] largest n_cell, [4] largest n_part, [5] groups
                                      beyond their slots (otoo_walk_single), then scratch */
} otoo_dev_walk;

/* Length of otoo_dev_walk.totals for n_groups groups. */
int64_t otoo_walk_totals_len(int64_t n_groups);

/* Pass 1 of the device walk: every group walks the tree once and
   groups[g] (device, n_groups records) receives first, count, n_cell,
   n_part, eps2, the centre of the particles' box, theta and sys = 0;
   list_off is the exclusive prefix sum of n_cell + n_part in group order.
   totals[0..2] = list entries, sum of count * (n_cell + n_part), sum of
   count * n_cell.  Asynchronous on stream; clears the status word. */
int otoo_walk_count(const otoo_dev_walk* walk, otoo_group* groups, void* stream);

/* Pass 2: walks again and writes each group's entries at list[list_off]:
   n_cell cell entries (source index n_part + k), then n_part particle
   entries.  list: device, capacity entries; when totals[0] > capacity the
   call writes no entry and sets the status word (checked by
   otoo_walk_check_status). */
int otoo_walk_fill(const otoo_dev_walk* walk, const otoo_group* groups, int32_t* list, int64_t capacity,
                   void* stream);

/* The walk in one pass (the steady state of a time loop, where the list
   sizes of the previous step bound the next): like otoo_walk_count, but each
   group's entries go straight to its fixed slot of slots (device, n_groups *
   (cell_cap + part_cap) int32), and the slots are the list.  Slot g starts
   at S g, S = cell_cap + part_cap; its cells are written backwards from
   S g + cell_cap - 1, its particles forwards from S g + cell_cap, so the
   group's entries lie contiguous, cells (in the reverse of the order
   otoo_walk_fill writes them) then particles, at list_off = S g + cell_cap -
   n_cell.  otoo_force and otoo_sph_density take slots as their list with
   n_list = n_groups S; no offsets are scanned.  totals[5] counts the groups
   with more entries than their slot: their entries are cut, their counts
   stay exact and their list_off is -1 (the force kernels reject it); walk
   again with otoo_walk_count and otoo_walk_fill.  Errors: OTOO_EINVAL
   (arguments, slot sizes below 1 or S above INT32_MAX).

   otoo_walk_compact copies the slots of a single pass into a dense list in
   group order, exactly what otoo_walk_count + otoo_walk_fill write (cells
   back in walk order), and rewrites groups[g].list_off to the dense offsets.
   list: device, capacity entries; nothing is copied (status word set) when
   totals[5] > 0 or totals[0] > capacity.  Asynchronous on stream. */
int otoo_walk_single(const otoo_dev_walk* walk, otoo_group* groups, int32_t* slots, int64_t cell_cap,
                     int64_t part_cap, void* stream);
int otoo_walk_compact(const otoo_dev_walk* walk, otoo_group* groups, const int32_t* slots, int64_t cell_cap,
                      int64_t part_cap, int32_t* list, int64_t capacity, void* stream);

/* The walk fused with the FP32 force (Section III-D: the paper's GPU kernel
   walks the tree for each group of particles and evaluates the interactions
   it finds, with no interaction list in memory).  One warp per group walks as
   otoo_walk_count does (same acceptance decisions) and evaluates each tile of
   accepted cells or leaf particles as soon as it is complete, with the pair
   arithmetic of otoo_force's packed FP32 form (centre-relative FP32 pairs,
   per-tile Kahan sums, FP64 outputs).
   walk: as for otoo_walk_count (OTOO_MAC_THETA or OTOO_MAC_SW; every group at
   most 32 * iblock particles, larger groups get no output and set the status
   word).  quad: device, [n_cell] quadrupoles as otoo_tree_device_arrays
   writes them, or NULL for monopole cells.  perm: device, [n_part] tree ->
   caller order (NULL: tree order).  split: device scratch, 8 * (n_part +
   n_cell) floats (the per-step float pairs of the positions).  iblock:
   targets per lane, 1, 2 or 4.  accel: device, [n_part][3]; pot: device,
   [n_part] (groups skipped by a negative per-group angle are not written).
   totals[0..4] as otoo_walk_count: list entries, interactions, cell
   interactions, largest n_cell and n_part.  Asynchronous on stream; errors
   of the walk or a group too large for iblock are reported by
   otoo_walk_check_status.  Errors: OTOO_EINVAL (arguments, OTOO_MAC_SPH),
   OTOO_ECUDA. */
int otoo_walk_force(const otoo_dev_walk* walk, const otoo_quad* quad, const int64_t* perm, float* split,
                    int32_t iblock, double* accel, double* pot, void* stream);

/* Reads the walk's status word after a sync: OTOO_EDEVICE when a record
   failed its bounds check, a group's stack overflowed, the two passes
   disagreed, or the list did not fit. */
int otoo_walk_check_status(const otoo_dev_walk* walk, void* stream);

/* Work items on the device with the rules of otoo_make_plan (the same
   items, splits and slot numbers; launch order: descending cost class
   instead of a sort, which changes no result).  groups: device records of
   otoo_walk_count.  Scratch: plan_scratch, >= otoo_plan_scratch_ints
   (n_groups) int32 (device).  plan_totals: device int64 [4] = items,
   splits, slots, n_crit_max, written by otoo_plan_count; the caller reads
   them (after a sync) to size items [plan_totals[0]], splits
   [plan_totals[1]] and the force step's partial scratch (plan_totals[2] *
   4 * plan_totals[3] doubles).  otoo_plan_fill writes nothing beyond the
   capacities it is given (status bit set in counter[1] instead). */
int64_t otoo_plan_scratch_ints(int64_t n_groups);
int otoo_plan_count(const otoo_group* groups, int32_t n_groups, const otoo_tune* tune, int32_t* plan_scratch,
                    int64_t* plan_totals, void* stream);
int otoo_plan_fill(const otoo_group* groups, int32_t n_groups, const otoo_tune* tune, int32_t* plan_scratch,
                   const int64_t* plan_totals, otoo_item* items, int64_t items_capacity, otoo_split* splits,
                   int64_t splits_capacity, uint32_t* counter, void* stream);

/* ---- the tree built on the device ------------------------------------------------
   Section III-B (root cube, keys, sort, cells) and III-C (cell properties) on
   the GPU, writing the device walk's and the force step's inputs in place.
   The root cube, grid coordinates, Hilbert keys, the stable (key, index)
   sort and the cell cubes use the host build's operations, so the particle
   order, the cells (as particle ranges with their levels), their cubes and
   the groups equal otoo_build_tree's; cells are numbered level by level
   (children consecutive), and the moments (mass, centre of mass,
   quadrupole, B_2, b_max) are combined bottom-up, equal to the host's direct
   sums to rounding.  The SPH radius of a cell (OTOO_MAC_SPH) is an FP32
   upper bound on the host's: larger by at most about 2^-20 relative plus
   the FP32 rounding of the positions, never smaller. */
typedef struct otoo_devtree {
    /* in */
    int64_t n_part;                /* particles (>= 1) */
    int64_t cap_cell;              /* capacity of the cell arrays below */
    int32_t leaf_size, n_crit;     /* as in otoo_params */
    int32_t use_quad, mac;         /* quadrupoles stored or zero; OTOO_MAC_THETA / _SW / _SPH */
    double delta, m_limit;         /* OTOO_MAC_SW: the walk records' r_b */
    const float* h_sph;            /* OTOO_MAC_SPH: device [n_part], caller order */
    /* out (host values) */
    int64_t n_cell, n_groups;      /* n_cell = -1 when cap_cell was too small */
    int32_t depth, pad;
    double root_lo[3], root_side;
    /* device arrays, caller-owned */
    otoo_src* src;                 /* [n_part + cap_cell]: particles in tree order, then cells */
    otoo_quad* quad;               /* [cap_cell] */
    otoo_wcell* cell;              /* [cap_cell] walk records */
    otoo_wcell64* cell64;          /* [cap_cell] */
    int32_t* group_first;          /* [n_part] */
    int32_t* group_count;          /* [n_part] */
    int64_t* perm;                 /* [n_part] caller index of each tree particle */
    int32_t* cell_level;           /* [cap_cell] level of each cell (0 = root) */
    uint32_t* status;              /* scratch, >= 2 uint32 */
} otoo_devtree;

/* Bytes of device scratch otoo_devtree_build needs (16-byte aligned). */
int64_t otoo_devtree_scratch_bytes(int64_t n_part, int64_t cap_cell);

/* Builds the tree of pos (device [n_part][3] FP64, caller order) and mass
   (device [n_part] FP32 > 0) on stream and fills tree's device arrays and
   out fields; synchronises stream once per tree level (the host reads each
   level's cell count).  Errors: OTOO_EINVAL (sizes, NULL pointers, scratch
   too small or not 16-byte aligned, a non-finite position or a mass <= 0),
   OTOO_ENOMEM (more cells than cap_cell: n_cell = -1; call again with a
   larger capacity), OTOO_ECUDA. */
int otoo_devtree_build(const double* pos, const float* mass, otoo_devtree* tree, void* scratch,
                       int64_t scratch_bytes, void* stream);

/* ---- SPH density (Section II, Bounding Radius for SPH) ---------------------------
   rho_i = sum_j m_j W(|x_i - x_j|, h_j) (Eq. SPH_SUM with A = m) over lists
   made with OTOO_MAC_SPH (particles only), W the M4 cubic spline with
   support radius h: W = 8 / (pi h^3) w(q), q = r / h, w = 1 - 6 q^2 + 6 q^3
   (q <= 1/2), 2 (1 - q)^3 (1/2 < q < 1), 0 beyond; the source itself
   included.  sys: as for otoo_force, with a plan made for these lists (the
   quad, accel-related fields are not read; sys->split, 32-byte aligned,
   serves as scratch for 32 bytes per particle: its position as a float pair,
   m 8/(pi h^3) and 1/h); h: device [n_part] neighbour radii, caller order (the
   order sys->perm maps to); rho: device [n_part] FP64, written at perm[k]
   (tree order when perm is NULL); tune->iblock in {1, 2, 4} as in the plan.
   FP32 pair terms relative to the group centre, Kahan-compensated FP32 sums
   across 32-entry tiles and lane subsets, FP64 sums across list chunks.  Asynchronous on stream; bad items or list indices
   set the status word (otoo_check_status). */
int otoo_sph_density(const otoo_dev_system* sys, const float* h, double* rho, const otoo_tune* tune, void* stream);

/* FP64 brute-force density for chosen targets, the reference of the checks:
   rho[t] = sum over all j < n of m_j W(|x_i - x_j|, h_j), i = targets[t]
   (index into src and h, which are in the same order).  Device arrays: src
   [n] (particles only), h [n], targets [n_tgt] int64, rho [n_tgt] FP64,
   status one uint32 (bit 2: a target index out of range).  Asynchronous. */
int otoo_sph_direct(const otoo_src* src, const float* h, int64_t n, const int64_t* targets, int64_t n_tgt,
                    double* rho, uint32_t* status, void* stream);

/* ---- learned opening angle (multilayer perceptron 6-32-32-1) ---------------- */

#define OTOO_MLP_IN  6
#define OTOO_MLP_H   32
#define OTOO_MLP_NPARAM (OTOO_MLP_H * OTOO_MLP_IN + OTOO_MLP_H + OTOO_MLP_H * OTOO_MLP_H + OTOO_MLP_H + OTOO_MLP_H + 1)

/* Parameter vector layout (FP32 master weights, 1313 floats):
   W1 [32][6], b1 [32], W2 [32][32], b2 [32], w3 [32], b3 [1].
   Forward: h1 = tanh(W1 x + b1), h2 = tanh(W2 h1 + b2), y = w3 . h2 + b3.
   The forward kernel reads bf16 copies of the weights (bf16: device, 1313 uint16). */

/* y[r] = network(x[r]) for r < n_rows; x: device [n_rows][6] FP32; y: device
   [n_rows] FP32; wbf16: device bf16 parameters.  Asynchronous on stream. */
int otoo_mlp_predict(const uint16_t* wbf16, const float* x, float* y, int64_t n_rows, void* stream);

/* Floats of device scratch the gradient and training calls need for n_rows
   rows (one gradient partial per 128 rows). */
int64_t otoo_mlp_scratch_floats(int64_t n_rows);

/* Gradient of loss = (1/n) sum_r (y_r - target_r)^2 for the bf16 forward
   pass: grad device [1313] FP32, loss device [1] (may be NULL).  The sum over
   rows runs in a fixed order (deterministic).  scratch: device,
   otoo_mlp_scratch_floats(n_rows) floats. */
int otoo_mlp_grad(const uint16_t* wbf16, const float* x, const float* target, int64_t n_rows,
                  float* scratch, float* grad, float* loss, void* stream);

/* One training step on a batch: the gradient above, then one Adam step
   (Kingma & Ba: lr, beta1, beta2, eps_adam, step count t >= 1, bias-corrected)
   on the FP32 master weights w with moments m, v (device [1313] each); the
   bf16 copy is rounded from the new w (nearest even); the batch loss before
   the step goes to loss[0] (device, may be NULL). */
int otoo_mlp_train_step(float* w, uint16_t* wbf16, float* m, float* v, float* scratch,
                        const float* x, const float* target, int64_t n_rows, float lr,
                        float beta1, float beta2, float eps_adam, int32_t t, float* loss,
                        void* stream);

/* Round FP32 weights to the bf16 copy (round to nearest even). */
int otoo_mlp_to_bf16(const float* w, uint16_t* wbf16, int32_t n, void* stream);

/* Rows standardised for the network with the training set's statistics:
   out[r][k] = (x[r][k] - mean[k]) / std[k] in FP32 (the same arithmetic as
   otoo_learned_theta).  Device arrays x, out [n_rows][6], mean, std [6].
   x and out may be the same array.  Asynchronous on stream. */
int otoo_mlp_standardise(const float* x, int64_t n_rows, const float* mean, const float* std, float* out,
                         void* stream);

/* Per-group opening angle: x holds n_groups * n_theta rows, row (g, k) being
   group g's features with the angle theta_grid[k] (grid increasing).
   theta_out[g] = the largest theta_grid[k] whose prediction y(g, k) <= the
   group's target (log10_target_per_group[g], or log10_target when that array
   is NULL), theta_grid[0] when none qualifies, fallback when any prediction
   of the group is not finite.  Device arrays, async on stream. */
int otoo_select_theta(const uint16_t* wbf16, const float* x, const float* theta_grid,
                      int32_t n_theta, int64_t n_groups, float log10_target,
                      const float* log10_target_per_group, float fallback, float* theta_out,
                      void* stream);

/* The learned opening angle from raw list statistics, every step on the
   device (the library's replacement of the paper's accuracy control, the
   Delta of the absolute MAC, Section II-B): per group g of a base walk at
   theta0 with statistics feat[g] (otoo_group_features, 5 floats) and count[g]
   particles,
     1. range: a group whose statistics are not finite or lie outside the
        training range [lo, hi] takes the fallback angle;
     2. budget: y0 = network(standardised (feat[g], theta0)) is its predicted
        log10 error at theta0, L = 2^feat[g][0] its list length; its weight is
        w = 10^(alpha y0 + beta log10 L), and its target
          e_g = lambda w,  lambda = calib target_rms / sqrt(sum n w^2 / sum n)
        over the groups in range (n = count), so that the particle-weighted
        RMS of the targets is calib * target_rms.  With a group error
        ~ c theta^k and a list length ~ theta^-3, the targets that minimise
        the interactions at a fixed particle-weighted RMS have alpha =
        3 / (2k + 3), beta = k / (2k + 3); alpha = beta = 0 gives every
        group the same target;
     3. choice: theta_out[g] = the largest grid[k] whose prediction
        network(standardised (feat[g], grid[k])) <= log10 e_g, grid[0] when
        none; the fallback when a prediction is not finite.
   Standardised = (x - mean) / std per input.  Device arrays: feat
   [n_groups][5], count [n_groups], grid [n_theta] (increasing), scratch
   otoo_learned_theta_scratch_floats(n_groups) floats (8-byte aligned),
   log10_target [n_groups] (may be NULL; NaN for groups out of range),
   theta_out [n_groups].  FP32 network and targets, FP64 sums in a fixed
   order (deterministic).  Asynchronous on stream. */
typedef struct otoo_theta_net {
    const uint16_t* wbf16;         /* device [OTOO_MLP_NPARAM] bf16 weights */
    const float* mean;             /* device [OTOO_MLP_IN] input means of the training rows */
    const float* std;              /* device [OTOO_MLP_IN] their standard deviations (> 0) */
    const float* lo;               /* device [OTOO_MLP_IN - 1] training range of the statistics, or */
    const float* hi;               /* NULL (both) for no range check */
} otoo_theta_net;

typedef struct otoo_theta_rule {
    float theta0;                  /* angle of the base walk the statistics come from (> 0) */
    float target_rms;              /* particle-weighted RMS relative acceleration error aimed at */
    float calib;                   /* calibration of the network: the groups aim at calib * target_rms */
    float alpha, beta;             /* budget exponents (0, 0: equal targets) */
    float fallback;                /* angle for groups out of range or with a non-finite prediction */
} otoo_theta_rule;

int64_t otoo_learned_theta_scratch_floats(int64_t n_groups);
int otoo_learned_theta(const otoo_theta_net* net, const otoo_theta_rule* rule, const float* feat,
                       const int32_t* count, int64_t n_groups, const float* grid, int32_t n_theta, float* scratch,
                       float* log10_target, float* theta_out, void* stream);

/* Training labels of the learned angle: per group g, the RMS over its
   targets [group_off[g], group_off[g + 1]) of the relative acceleration
   error |acc - ref| / |ref| (acc, ref: device [n][3] FP64, ref the FP64
   direct sum), as log10_rms[g] = log10(max(rms, floor_value)) (device
   [n_groups] FP32).  group_off: device [n_groups + 1], non-decreasing; an
   empty or negative range sets status (device, one uint32) and gives NaN.
   One warp per group, sums in a fixed order.  Asynchronous on stream. */
int otoo_group_rms_error(const double* acc, const double* ref, const int64_t* group_off, int64_t n_groups,
                         float floor_value, float* log10_rms, uint32_t* status, void* stream);

const char* otoo_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* OTOO_H */
