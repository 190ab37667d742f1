/*
 * sl.h -- C ABI of the GB300 semi-Lagrangian foot / locate / P1 library.
 *
 * One semi-Lagrangian step (Cacace & Ferretti, Sec. 1 and Algorithm 2) maps
 * the node values V^n of a triangulation of the unit square to V^{n+1}:
 *
 *     v_i^{n+1} = I[V^n]( X^Delta(x_i, t_{n+1}; t_n) )                (Eq. 3)
 *
 * with the Euler foot X = x_i - dt f(x_i, t_{n+1}) (Eq. 4), clipped to the
 * square where it leaves it, located by a barycentric walk over the triangle
 * adjacency (Sec. 2.2, Algorithm 1) that starts from the triangle found for
 * the same node at the previous step (walk strategy (b), Sec. 3), and
 * evaluated by P1 interpolation with the barycentric coordinates of Eq. 6
 * (Remark 1 of Sec. 2.2).
 *
 * Conventions shared by every entry point:
 *   - Every function returns an sl_status; nothing throws across the ABI.
 *     sl_last_error() returns a thread-local message for the last failure.
 *   - "host" pointers are ordinary CPU memory; "device" pointers are CUDA
 *     device memory of the current device.  The caller keeps ownership of
 *     everything it passes; host inputs are copied before the call returns.
 *   - Indices are 0-based and local to their problem (the paper's lists are
 *     1-based, Sec. 3).
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Work is enqueued asynchronously on it; errors found while
 *     launching are returned at once, conditions found by the kernels (a walk
 *     that gave up) are reported by sl_mesh_status() or sl_run().
 *   - A mesh handle may be used by one stream at a time.
 */
#ifndef SL_H
#define SL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SL_OK = 0,
    SL_E_ARG = 1,          /* invalid argument (null pointer, bad size, NaN/Inf parameter) */
    SL_E_MESH = 2,         /* malformed mesh (see sl_mesh_create) */
    SL_E_NOMEM = 3,        /* host or device allocation failed */
    SL_E_CUDA = 4,         /* a CUDA runtime call failed */
    SL_E_WALK_LIMIT = 5,   /* some walk exceeded its hop cap and its fallback */
    SL_E_STATE = 6         /* call not valid in the handle's current state */
} sl_status;

typedef enum { SL_FP64 = 0, SL_FP32 = 1 } sl_precision;

typedef enum { SL_CURVE_NONE = 0, SL_CURVE_HILBERT = 1, SL_CURVE_MORTON = 2 } sl_curve;

/* Advecting fields f(x, t); p = sl_problem.p.
 *   ZERO      f = 0
 *   AFFINE    f_x = p0 + p1 x + p2 y + p3 t,  f_y = p4 + p5 x + p6 y + p7 t
 *   ROTATION  f = p0 (p2 - y, x - p1)
 *   SWIRL     f = cos(pi t / p0) (sin^2(pi x) sin(2 pi y), -sin^2(pi y) sin(2 pi x))
 *   FOURIER8  psi = sum_{m<8} a_m cos(2 pi t + phi_m) sin(k_m pi x) sin(l_m pi y),
 *             f = (d psi/dy, -d psi/dx); (k_m, l_m, a_m, phi_m) = p[4m .. 4m+3]
 *   PAPER     f = (cos(p0 r + p1 t), sin(p0 r + p1 t)), r = |x - (p2, p3)|:
 *             the test field of the paper's Sec. 4 (C0 = p0, C1 = p1). */
typedef enum {
    SL_FIELD_ZERO = 0,
    SL_FIELD_AFFINE = 1,
    SL_FIELD_ROTATION = 2,
    SL_FIELD_SWIRL = 3,
    SL_FIELD_FOURIER8 = 4,
    SL_FIELD_PAPER = 5
} sl_field_kind;

#define SL_NPARAMS 48

/* One problem's field and time step.  Host memory. */
typedef struct {
    int32_t kind;          /* sl_field_kind */
    int32_t reserved;      /* must be 0 */
    double dt;             /* time step (> 0, finite) */
    double p[SL_NPARAMS];  /* field parameters (finite) */
} sl_problem;

/* Per-node flag bits written to sl_debug.flags */
enum {
    SL_NODE_CLIPPED = 1,      /* the Euler foot left the square and was clipped */
    SL_NODE_DEGENERATE = 2,   /* the foot lies on an edge line of its triangle */
    SL_NODE_EXACT = 4,        /* an orientation sign needed the exact stage */
    SL_NODE_FALLBACK = 8,     /* the walk hit its hop cap and used the fallback walk */
    SL_NODE_WALK_LIMIT = 16,  /* the fallback failed too: the value is not valid */
    SL_NODE_RANGE = 32,       /* a coordinate outside the exact predicate's range */
    SL_NODE_EXCLUDED = 64,    /* SL_OPT_OUTSIDE = 1: the Euler foot left the square, so the node
                                 was excluded (V^{n+1}_i = V^n_i, no walk, T^0_i unchanged) */
    SL_NODE_PRECISE = 128     /* double-float kernel: the value was evaluated in FP64 because V^n
                                 is steep in the located triangle (SL_OPT_PRECISE) */
};

typedef struct sl_mesh sl_mesh;   /* opaque; owns device mesh arrays and T^0 */

/* Optional per-node outputs of sl_step (device pointers, each may be NULL).
 * Arrays are indexed by node in the mesh's current numbering (all problems
 * concatenated). */
typedef struct {
    double *feet;     /* 2N doubles: the clipped foot (x, y) of every node, rounded to double */
    int32_t *tri;     /* N: located triangle, global index in current numbering */
    int32_t *moves;   /* N: walk hops (0 if the start triangle contains the foot) */
    uint8_t *flags;   /* N: SL_NODE_* bits */
    double *feet_lo;  /* 2N doubles: the exact rest of the foot, so that feet + feet_lo (summed
                         exactly, per coordinate) is the point the kernel located.  The
                         double-float kernel holds a foot as a pair of floats, which one double
                         cannot always represent; the plain FP64 and the FP32 kernels write 0. */
} sl_debug;

/* Counters accumulated on the device by sl_step / sl_run when enabled with
 * sl_mesh_set_option(SL_OPT_STATS, 1).  Read with sl_mesh_stats(). */
typedef struct {
    uint64_t node_updates;   /* nodes stepped */
    uint64_t walk_moves;     /* total hops */
    uint64_t max_moves;      /* longest walk */
    uint64_t exact_tests;    /* orientation signs that needed the exact stage */
    uint64_t filter2_tests;  /* signs decided by the second (FP64) filter stage */
    uint64_t clipped;        /* feet clipped to the boundary */
    uint64_t fallbacks;      /* walks that switched to the fallback rule */
    uint64_t walk_limit;     /* walks that failed */
    uint64_t excluded;       /* nodes excluded (SL_OPT_OUTSIDE = 1); node_updates counts them too */
} sl_stats;

/* Tunable options (sl_mesh_set_option) */
typedef enum {
    SL_OPT_STATS = 0,        /* 0/1: accumulate sl_stats counters (default 0) */
    SL_OPT_WALK_CAP = 1,     /* hops before the fallback rule (default max(64, 4 (M+1))) */
    SL_OPT_KERNEL = 2,       /* 0 = auto (fast), 1 = plain FP64 kernel, 2 = fast kernel */
    SL_OPT_BLOCK = 3,        /* threads per block of the plain FP64 kernel (0 = auto) */
    /* 4 and 6 are not options (SL_E_ARG) */
    SL_OPT_CONFIG = 5,       /* launch configuration of the fast kernels, 0..5: threads per block x
                                blocks per SM the registers are sized for = 256x4, 256x3, 128x8,
                                128x9, 256x5, 128x12 (default 5) */
    SL_OPT_CONFIG_FIRST = 7, /* launch configuration for a step whose walks start at the initial
                                incident triangles (the first step after sl_mesh_create or
                                sl_mesh_reset_t0): long walks favour fewer resident warps (default 0) */
    SL_OPT_STRATEGY = 8,     /* start triangle of the walks (Sec. 3): 0 = strategy (b), the triangle
                                found at the previous step (default); 1 = strategy (a), the node's own
                                incident triangle at every step (T^0 is never overwritten); 2 = the
                                direct location of Sec. 4 on a structured Courant grid (one problem
                                of M x M cells, each split along its (l,m)-(l+1,m+1) diagonal, any
                                numbering; SL_E_ARG for other meshes): the walk starts at the triangle
                                the formula gives for the foot and corrects it if rounding put the
                                guess next door; 3 = strategy (c), the triangle just located for
                                the node's parent in a breadth-first spanning tree of the node
                                graph rooted at the node nearest (0.5, 0.5) (Sec. 3, 4): one launch
                                per tree level and step, no graph (sl_run's use_graph is ignored);
                                T^0_i holds the node's own foot triangle after each step.  Setting
                                it resets T^0 to the initial incident triangles (synchronises). */
    SL_OPT_OUTSIDE = 9,      /* feet that leave the square: 0 = clip them to the boundary (default);
                                1 = exclude the node, as the paper's experiments do (Sec. 4):
                                V^{n+1}_i = V^n_i, flag SL_NODE_EXCLUDED */
    SL_OPT_SPLIT = 10,       /* FP64 meshes, strategy (b), feet clipped: 0 = one fused kernel per
                                step (default); 1 = two passes per step: a lean pass finishes
                                every node whose foot is certainly inside its start triangle and
                                queues the others for the full kernel (fewer registers where the
                                feet move little).  Results are identical.  Never used for a step
                                from the initial start triangles.  sl_autotune sets it. */
    SL_OPT_ASYNC = 11,       /* 0 = sl_run synchronises the stream and returns the device status
                                (default); 1 = sl_run returns once its steps are enqueued when
                                stats is NULL, and the device status is read by the next
                                sl_mesh_status (or a synchronising sl_run).  Lets a caller queue
                                many runs back to back. */
    SL_OPT_PRECISE = 12,     /* FP64 meshes, double-float kernel: gradient bound G >= 0 (value
                                units per unit length; default 32; 0 = never).  The double-float
                                foot and barycentric coordinates carry about 2^-48 of rounding (a
                                foot moved by a few 2^-49), so a step's value is off by about
                                2^-46 |grad V|.  Where V^n in the located triangle is steeper
                                than G (max_k (v_k - v_3)^2 > G^2 den, den = twice its area), the
                                foot of an unclipped node, its barycentric coordinates (Eq. 6)
                                and the P1 value are evaluated again in FP64 from the double
                                coordinates, as the plain kernel does; the located triangle is
                                the same.  Scale G with the magnitude of V. */
    SL_OPT_RECORDS = 13,     /* half-edge walk records of the double-float kernel: 0 = 16-byte
                                records (default); 1 = 8-byte records where the mesh allows them
                                (every edge shorter than 2^17 grid units of 2^-24, about 2^-7,
                                and at most 44.7 M triangles), else 16-byte ones.  An 8-byte
                                record is one 64-bit gather per hop, which takes fewer L1
                                wavefronts for a warp's 32 scattered lanes, but more instructions
                                to unpack; sl_autotune measures both.  Results are identical.
                                Setting it rebuilds the records (synchronises). */
    SL_OPT_L2_WINDOW = 14,   /* 0 = off (default); 1 = in runs recorded as a CUDA graph, the
                                kernels mark the half-edge walk records as persisting in L2 (an
                                access-policy window of at most the device's window size, hit ratio
                                scaled to its persisting capacity, which this sets as the
                                context's persisting L2 limit; restored, and the persisting lines
                                reset, when the option goes back to 0 or the mesh is destroyed) */
    SL_OPT_PDL = 15          /* 1 = (default) in a sequence of steps (sl_run, sl_run_host), every
                                step kernel that follows a step kernel of the same sequence is
                                launched with programmatic stream serialization: its blocks may
                                start while the kernel before it finishes, compute their feet
                                (which need only the node coordinates and the field), and wait
                                for that kernel before they read T^0 or V^n.  0 = plain launches.
                                Results are identical.  No counterpart in the paper. */
} sl_option;

/*
 * sl_mesh_create -- validate a batch of triangulations and upload it.
 *
 * Builds the data of the paper's Sec. 3 (node list V, triangle list T,
 * neighbour list N with j_k the triangle across the edge opposite vertex
 * i_k, and the start-triangle list T^0, initialised to a random triangle
 * incident to each node) for `n_problems` independent meshes.
 *
 *   n_problems   >= 1
 *   node_off     host, n_problems+1 int64: problem p owns nodes
 *                [node_off[p], node_off[p+1]) of xy; node_off[0] = 0
 *   tri_off      host, n_problems+1 int64: the same for triangles
 *   xy           host, 2*N doubles (x, y) in [0,1]^2
 *   tri          host, 3*Nt int32 vertex indices local to the problem,
 *                counter-clockwise
 *   nbr          host, 3*Nt int32 or NULL: neighbour triangles local to the
 *                problem, nbr[3j+k] across the edge opposite tri[3j+k],
 *                -1 on the boundary; NULL = built here
 *   precision    SL_FP64 or SL_FP32 (FP32 stores coordinates rounded to
 *                nearest float; the caller's V buffers are then float)
 *   seed         selects the initial incident triangle of every node:
 *                T^0_i = the (h mod deg_i)-th incident triangle in ascending
 *                index, h = SplitMix64 value number i of `seed`
 *   out          receives the handle
 *
 * Returns SL_E_MESH for: an index out of range, a triangle that is not
 * strictly counter-clockwise (exact test), an edge shared by more than two
 * triangles or by two triangles with the same orientation, an inconsistent
 * supplied nbr, a boundary edge not lying on one side of the square, a node
 * outside the square or in no triangle, or a total area that is not 1;
 * SL_E_ARG for more than 2^31 - 1 nodes or 715 827 882 triangles (the fast
 * kernels number the edges of triangle t as 3 t + k in int32).
 */
sl_status sl_mesh_create(int32_t n_problems, const int64_t *node_off, const int64_t *tri_off,
                         const double *xy, const int32_t *tri, const int32_t *nbr,
                         int32_t precision, uint64_t seed, sl_mesh **out);

/*
 * sl_mesh_validate -- the host half of sl_mesh_create on its own: the same
 * arguments and checks, and the neighbour list and initial start triangles
 * it builds, without touching any GPU.
 *   nbr_out  host, 3*Nt int32 or NULL: neighbours, local to the problem, -1
 *            on the boundary (Sec. 3: j_k across the edge opposite i_k)
 *   t0_out   host, N int32 or NULL: initial T^0, local to the problem
 * Returns what sl_mesh_create would return for the mesh (SL_E_MESH, ...).
 */
sl_status sl_mesh_validate(int32_t n_problems, const int64_t *node_off, const int64_t *tri_off,
                           const double *xy, const int32_t *tri, const int32_t *nbr, uint64_t seed,
                           int32_t *nbr_out, int32_t *t0_out);

/*
 * sl_mesh_reorder -- renumber nodes and triangles along a space-filling
 * curve (per problem; problems keep their ranges).  Nodes are ordered by the
 * curve index of their position, triangles by that of their centroid; T, N
 * and T^0 are remapped so results are unchanged up to the permutation.
 * node_perm (host, N, may be NULL) receives new -> old node indices (local to
 * the problem), tri_perm (host, Nt, may be NULL) the same for triangles.
 * Must be called before the caller fills V buffers in the new numbering.
 */
sl_status sl_mesh_reorder(sl_mesh *m, int32_t curve, int32_t *node_perm, int32_t *tri_perm);

/*
 * sl_step -- one semi-Lagrangian step n -> n+1 for every node of every
 * problem (Eq. 3 with the Euler foot of Eq. 4 at t_{n+1} = (n+1) dt).
 *
 *   probs   host, n_problems entries
 *   v_in    device, N values V^n (double for SL_FP64, float for SL_FP32)
 *   v_out   device, N values V^{n+1}; must not alias v_in
 *   dbg     host struct of device pointers, or NULL
 * T^0 is updated in place to the located triangles (strategy (b)).
 */
sl_status sl_step(sl_mesh *m, const sl_problem *probs, int64_t n, const void *v_in, void *v_out,
                  const sl_debug *dbg, void *stream);

/*
 * sl_run -- n_steps steps from n0 (Algorithm 2's time loop).  `v` (device,
 * N values) holds V^{n0} on entry and V^{n0+n_steps} on return; `v_scratch`
 * (device, N values) is used for the ping-pong.  With use_graph != 0 the
 * steps are recorded once into a CUDA graph and replayed (the graph is kept
 * in the handle and reused while n0, n_steps, the buffers and the problems
 * are unchanged).  Synchronises the stream and returns the deferred device
 * status (SL_E_WALK_LIMIT if a walk failed).  stats may be NULL; with
 * SL_OPT_ASYNC = 1 and stats NULL it returns without synchronising.
 */
sl_status sl_run(sl_mesh *m, const sl_problem *probs, int64_t n0, int32_t n_steps, void *v,
                 void *v_scratch, int32_t use_graph, sl_stats *stats, void *stream);

/*
 * sl_run_host -- sl_run on HOST value buffers: copies V^{n0} (host, N values)
 * to device buffers owned by the handle, runs, copies V^{n0+n_steps} back
 * into the same host array, and synchronises.  Page-locked host memory makes
 * the copies asynchronous DMA; pageable memory works but is slower.
 */
sl_status sl_run_host(sl_mesh *m, const sl_problem *probs, int64_t n0, int32_t n_steps, void *v_host,
                      int32_t use_graph, sl_stats *stats, void *stream);

/* Limits of sl_step_noalloc's static scratch (see below). */
#define SL_NOALLOC_MAX_NODES (1 << 20)
#define SL_NOALLOC_MAX_PROBLEMS 256

/*
 * sl_step_noalloc -- the same step as sl_step for FP64 meshes (double values
 * in and out), performing no device allocation.  It always runs the fused
 * double-float kernel in the launch configuration sl_step would use for the
 * step: SL_OPT_KERNEL = 1 (the plain FP64 kernel) and SL_OPT_SPLIT do not
 * apply to it (the split form gives the same results).  The paper has no
 * counterpart: this exists for callers that cannot allocate device memory
 * while they step -- code running inside a host application whose caching
 * allocator owns the device memory, callbacks that must not synchronise the
 * device (cudaMalloc and cudaFree do), or programs with a fixed memory
 * budget reserved at start-up.
 *
 *   probs   host, n_problems entries (at most SL_NOALLOC_MAX_PROBLEMS)
 *   v_in    device, N doubles V^n
 *   v_out   device, N doubles V^{n+1}; must not alias v_in
 * The mesh must have at most SL_NOALLOC_MAX_NODES nodes (over all problems)
 * and must be an FP64 mesh; otherwise SL_E_ARG with a message naming the
 * limit.  Fields with node tables (SWIRL, PAPER, FOURIER8) need the tables
 * already built for these exact problems by an earlier sl_step / sl_run call
 * on the mesh (that call allocates them); otherwise SL_E_STATE.
 *
 * All scratch lives in one library-owned static device array per GPU
 * (8 MiB of value pairs + 16 KiB of per-problem constants), held by every
 * GPU that loads the library until the process exits.  The step's constants
 * reach that array in the parameters of a small kernel; no host buffer of
 * the call is read after it returns.  The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress); make
 * that first call before any stream capture.  Every call on a device shares
 * the array and overwrites what it uses, so calls that overlap on the GPU
 * (other streams, other meshes) race on it: serialise them.  T^0 is updated
 * in place as in sl_step; device conditions are reported by sl_mesh_status.
 */
sl_status sl_step_noalloc(sl_mesh *m, const sl_problem *probs, int64_t n, const double *v_in, double *v_out,
                          void *stream);

/* Result of sl_autotune: chosen launch configurations and the measured
 * times per configuration (milliseconds; -1 where not measured). */
#define SL_TUNE_MAX_CONFIGS 8
typedef struct {
    int32_t config_first;                 /* chosen SL_OPT_CONFIG_FIRST */
    int32_t config_rest;                  /* chosen SL_OPT_CONFIG */
    int32_t n_configs;                    /* configurations measured */
    int32_t split;                        /* chosen SL_OPT_SPLIT (FP64 meshes) */
    float first_ms[SL_TUNE_MAX_CONFIGS];  /* one step from the initial start triangles */
    float rest_ms[SL_TUNE_MAX_CONFIGS];   /* mean of the later steps */
    float split_ms[SL_TUNE_MAX_CONFIGS];  /* [0]: mean of the later steps, split (FP64 meshes) */
    int32_t records;                      /* chosen SL_OPT_RECORDS */
    float compact_first_ms;               /* the chosen configurations with 8-byte records: first */
    float compact_rest_ms;                /* ... and later steps (split if chosen); -1: not eligible */
    int32_t curve;                        /* sl_autotune_layout: chosen numbering (SL_CURVE_NONE = as
                                             given at the call), else -1 */
    float curve_ms[3];                    /* sl_autotune_layout: first step + probe_steps later steps
                                             per sl_curve value (-1: not tried) */
} sl_tune;

/*
 * sl_autotune -- choose the launch configurations of the fast kernels for
 * this mesh and these problems by measurement: for every configuration, one
 * step from the initial start triangles and `probe_steps` later steps are
 * timed with CUDA events on `stream`; the fastest configuration of each
 * phase becomes SL_OPT_CONFIG_FIRST and SL_OPT_CONFIG.  On FP64 meshes the
 * later steps are also timed split (SL_OPT_SPLIT = 1, whose passes have a
 * launch shape of their own), and the faster form is kept; then, where the
 * mesh allows 8-byte walk records, the chosen configurations are timed with
 * them, and they are kept (SL_OPT_RECORDS = 1) if a 50-step run (the first
 * step and 49 later ones) is faster.  v (device, N values,
 * V^0) and v_scratch (device, N values) are used as in sl_run; v, T^0 and
 * the statistics counters are restored before returning (the call
 * synchronises and allocates temporary device buffers).  No counterpart in
 * the paper: it tunes the launch shape of the fused step.
 */
sl_status sl_autotune(sl_mesh *m, const sl_problem *probs, int32_t probe_steps, void *v, void *v_scratch,
                      sl_tune *out, void *stream);

/*
 * sl_autotune_layout -- choose the numbering of nodes and triangles by
 * measurement, then tune as sl_autotune.  For each layout in `curves` (bit c
 * set = try sl_curve c; SL_CURVE_NONE = the numbering at the call), the mesh
 * is renumbered (per problem, as sl_mesh_reorder) and one step from the
 * initial start triangles plus `probe_steps` later steps are timed in the
 * current launch configuration; the fastest layout is kept.  Nodes that are
 * neighbours in space are neighbours in memory along a space-filling curve
 * (Hilbert or Morton), which decides how many sectors a warp's gathers
 * touch.  v (device, N values of V^0 in the numbering at the call) is
 * permuted in place to the kept numbering; node_perm / tri_perm (host, N /
 * Nt int32, or NULL) receive new -> old indices relative to the numbering
 * at the call, local to each problem.  T^0 follows the renumbering.  out
 * receives sl_autotune's results and the curve fields.  Synchronises;
 * allocates temporary device buffers.  No counterpart in the paper (its
 * meshes keep the Triangle library's numbering).
 */
sl_status sl_autotune_layout(sl_mesh *m, const sl_problem *probs, int32_t probe_steps, int32_t curves, void *v,
                             void *v_scratch, int32_t *node_perm, int32_t *tri_perm, sl_tune *out, void *stream);

/*
 * sl_probe_gather -- the memory-system ceiling of a later step (FP64
 * meshes): one kernel that makes exactly the memory accesses of a step in
 * which every foot stays in its start triangle -- the node's coordinate pair
 * and start state, the start triangle's three vertex pairs and three values,
 * one value written -- with no arithmetic beyond summing what it read.  It
 * runs over the mesh's current T^0, in the launch shape of the settle pass,
 * once untimed and then `reps` times (1..1000) timed with CUDA events on
 * `stream`; *ms_out receives the mean time per launch.  v (device, N
 * doubles) is read as (hi, lo) float pairs; v_scratch (device, N doubles) is
 * overwritten with meaningless values; T^0 and the statistics are not
 * touched.  Synchronises.  No counterpart in the paper: it measures the
 * effective gather roofline a step of this mesh is held to.
 */
sl_status sl_probe_gather(sl_mesh *m, const void *v, void *v_scratch, int32_t reps, float *ms_out, void *stream);

/*
 * sl_mesh_get_t0 / sl_mesh_set_t0 -- export / import the start-triangle list
 * T^0 of Sec. 3 (Algorithm 1 reads T^0_i as the walk's first triangle and,
 * in strategy (b), stores the foot triangle T^f_i there).  t0_dev: device,
 * N int32, global triangle indices in the current numbering, written (get)
 * or read (set) on `stream`; the caller owns it.  With V^n this is the whole
 * state of a run, so a run can stop and resume bitwise.  set validates every
 * entry (SL_E_ARG if one is not a triangle of its node's problem; it copies
 * T^0 through the host and synchronises) and refreshes the start-state cache.
 */
sl_status sl_mesh_get_t0(const sl_mesh *m, int32_t *t0_dev, void *stream);
sl_status sl_mesh_set_t0(sl_mesh *m, const int32_t *t0_dev, void *stream);

/* Put T^0 back to the initial start triangles chosen by sl_mesh_create (in
 * the current numbering), on the device, asynchronously on `stream`: the
 * next step then starts every walk from a triangle incident to its node, as
 * the first step of a run does (Sec. 3: strategies (a) and (b) coincide on
 * the first step). */
sl_status sl_mesh_reset_t0(sl_mesh *m, void *stream);

/*
 * sl_mesh_status -- synchronise `stream` and return (and clear) the deferred
 * device status: SL_E_WALK_LIMIT when a walk exceeded its hop cap and its
 * fallback (reading c9: the paper assumes Delaunay meshes, on which the walk
 * of Algorithm 1 always ends), SL_E_ARG when a coordinate fell outside the
 * exact predicate's range, SL_OK otherwise.
 */
sl_status sl_mesh_status(sl_mesh *m, void *stream);

/*
 * sl_mesh_stats -- read (and with reset != 0, clear) the device counters of
 * sl_stats (out: host); synchronises `stream`.  The hop counts are the walk
 * steps of Algorithm 1 that the paper measures (Sec. 2.2, Sec. 4: mean moves
 * per located point); the other counters have no counterpart in the paper.
 */
sl_status sl_mesh_stats(sl_mesh *m, sl_stats *out, int32_t reset, void *stream);

/*
 * sl_mesh_set_option -- set one sl_option (values and ranges documented with
 * the enum; SL_E_ARG for an unknown option or a value out of range).
 * SL_OPT_STRATEGY selects the start strategies of Sec. 3 and the direct
 * location of Sec. 4, SL_OPT_OUTSIDE the exclusion of Sec. 4; the others are
 * launch and instrumentation settings with no counterpart in the paper.
 * Host only, except SL_OPT_STRATEGY, which resets T^0 and synchronises.
 */
sl_status sl_mesh_set_option(sl_mesh *m, int32_t option, int64_t value);

/* sl_mesh_get_option -- the current value of an sl_option (value: host),
 * except SL_OPT_RECORDS, for which it gives the size in bytes of the
 * half-edge walk records the mesh uses (8 or 16).  SL_E_ARG for an unknown
 * option.  No counterpart in the paper. */
sl_status sl_mesh_get_option(const sl_mesh *m, int32_t option, int64_t *value);

/* sl_mesh_info -- the sizes of the handle (host outputs, each may be NULL):
 * nodes and triangles over all problems, problems, precision.  No
 * counterpart in the paper. */
sl_status sl_mesh_info(const sl_mesh *m, int64_t *n_nodes, int64_t *n_tri, int32_t *n_problems,
                       int32_t *precision);

/* sl_mesh_export -- the mesh in its current numbering: the node list V, the
 * triangle list T and the neighbour list N of Sec. 3 (host arrays owned by
 * the caller: xy 2N doubles, tri 3Nt int32 local vertex indices, nbr 3Nt
 * int32 local neighbours, -1 on the boundary; each may be NULL). */
sl_status sl_mesh_export(const sl_mesh *m, double *xy, int32_t *tri, int32_t *nbr);

/* sl_mesh_destroy -- free the handle and every device buffer it owns
 * (NULL is ignored).  No counterpart in the paper. */
void sl_mesh_destroy(sl_mesh *m);

/* sl_last_error -- the calling thread's message for its last failed call
 * (valid until its next call).  No counterpart in the paper. */
const char *sl_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
