/*
 * cem.h -- C ABI of the GB300 crack element method (CEM) library.
 *
 * The library advances the explicit ES-T-FEM time step of the 3D crack
 * element method (arxiv 2508.04076) on a linear-tetrahedron mesh held in GPU
 * memory, evaluates the energy release rate of every crack-front element and
 * splits elements whose rate exceeds Gc.  All arithmetic of the step runs in
 * the library's own sm_103a CUDA kernels.
 *
 * Conventions shared by every entry point
 *   - Every function returns an int status: CEM_OK (0) or a negative CEM_E*
 *     code.  cem_last_error() returns a message for the last failure on a
 *     context (a static string owned by the context, valid until the next
 *     call on it).
 *   - Host arrays passed in are read during the call and copied; the caller
 *     keeps ownership.  Outputs go to caller-owned host buffers.
 *   - Device memory is obtained through the allocator in cem_mesh_desc (or
 *     cudaMalloc when none is given) in cem_mesh_create, and by cem_adjoint
 *     for its working memory (released before it returns); cem_step never
 *     allocates.  Every allocation of the context is released by cem_destroy.
 *   - All device work is queued on the stream given at creation.  cem_step
 *     synchronises that stream once per step while crack-front elements exist
 *     (to learn whether any element splits); cem_energy, cem_crack_state and
 *     cem_get_field return after their results are on the host.
 *   - A context is not thread-safe; use one host thread per context.
 *   - Node arrays are returned in the library's canonical order: the input
 *     nodes first, then one node per (cut original edge, endpoint side) in
 *     ascending (edge id, side) order, where original edge ids enumerate the
 *     input mesh's edges by ascending (smaller node id, larger node id).
 *   - Element local numbering: local edge l joins local nodes
 *     (0,1),(0,2),(0,3),(1,2),(1,3),(2,3); local face f is the face opposite
 *     local node f.  An element given with negative signed volume has its
 *     local nodes 2 and 3 swapped on input (side masks are permuted alike).
 */
#ifndef CEM_H
#define CEM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define CEM_OK          0
#define CEM_EINVAL     -1   /* bad argument or malformed mesh                        */
#define CEM_ENOMEM     -2   /* the allocator returned NULL                           */
#define CEM_ECUDA      -3   /* a CUDA runtime call failed                            */
#define CEM_ECAPACITY  -4   /* split or storage capacity exhausted (see cem_step)    */
#define CEM_ENONFINITE -5   /* a non-finite displacement was produced               */
#define CEM_ETIMEOUT   -6   /* a bounded device wait gave up (see cem_set_wait_limit)*/
#define CEM_ESTATE     -7   /* call not valid in the context's current state        */

/* precision of the force evaluation */
#define CEM_FP64   0        /* every quantity in FP64                                */
#define CEM_MIXED  1        /* FP32 element strains, edge stresses and element forces; */
                            /* FP64 node state, integration, energies and G test      */

/* fields for cem_get_field */
#define CEM_FIELD_U 0       /* displacement u                                         */
#define CEM_FIELD_V 1       /* velocity v                                             */
#define CEM_FIELD_A 2       /* acceleration a                                         */
#define CEM_FIELD_X 3       /* reference coordinates X                                */

/* crack patterns reported by cem_crack_state (Sec. 3, Fig. 5) */
#define CEM_PATTERN_I  1    /* quadrilateral G1 G2 G4 G3: two nodes on each side      */
#define CEM_PATTERN_II 2    /* triangle G1 G2 G6: one node cut off                    */

/* element type (cem_mesh_desc.elem_type) */
#define CEM_ELEM_TET4 0         /* linear tetrahedra, ES-T-FEM (Sec. 2.2); the crack path */
#define CEM_ELEM_HEX8 1         /* trilinear hexahedra, ES-H-FEM (Sec. 2.2), fixed       */
                                /* topology (no crack patterns: those of Sec. 3 for      */
                                /* hexahedra are defined only by figures)                */

/* split rule (cem_mesh_desc.split_mode) */
#define CEM_SPLIT_SUBDIVIDE  0  /* the split element is replaced by sub-tetrahedra on    */
                                /* both sides of its crack (its remainder keeps working) */
#define CEM_SPLIT_DEACTIVATE 1  /* the split element only leaves the computation         */
                                /* (literal wording of Sec. 1 and the conclusion)        */

/* traction of the energy release rate (cem_mesh_desc.g_variant), Eqs. 17-18 */
#define CEM_G_PRINCIPAL 0       /* s = sigma_1 |p_1 . n| (principal-stress vector)        */
#define CEM_G_NORMAL    1       /* s = n . sigma n (normal traction of the edge stress)   */

/* Device allocator hooks.  alloc returns a device pointer of at least `bytes`
 * bytes (256-byte aligned) or NULL; free releases it.  `stream` is the
 * context's stream.  Both are called only inside cem_mesh_create,
 * cem_adjoint, cem_autotune (once per context) and cem_destroy. */
typedef void* (*cem_alloc_fn)(size_t bytes, void* stream, void* user);
typedef void  (*cem_free_fn)(void* ptr, void* stream, void* user);

/* Mesh, load and notch description for cem_mesh_create (host pointers). */
typedef struct cem_mesh_desc {
    int64_t        n_nodes;      /* N > 0                                              */
    int64_t        n_tets;       /* T > 0                                              */
    const double*  X;            /* N x 3 row-major reference coordinates [m]          */
    const int32_t* tets;         /* T x 4 node ids of linear tetrahedra                */
    int64_t        n_tfaces;     /* F >= 0 traction faces                              */
    const int32_t* tfaces;       /* F x tface_nodes node ids                           */
    const double*  tvec;         /* F x 3 traction vector of each face [Pa]; the load  */
                                 /* t*A/3 goes to each face node (Sec. 2.2, Eq. 12)    */
    int64_t        n_notch;      /* K >= 0 pre-split (notch) elements                  */
    const int32_t* notch_tet;    /* K element ids, distinct                            */
    const uint8_t* notch_side;   /* K 4-bit masks over local nodes naming the two      */
                                 /* sides of the notch crack (not 0, not 15)           */
    int32_t        precision;    /* CEM_FP64 or CEM_MIXED                              */
    double         dt;           /* > 0: fixed step [s]; <= 0: cfl_factor * h_min /   */
                                 /* (2 c_d) (see cem_set_material)                     */
    double         cfl_factor;   /* used when dt <= 0; <= 0 means 0.5                  */
    int32_t        split_enabled;/* 0: fixed topology after the notch; 1: CEM splitting*/
    int64_t        split_capacity; /* max original elements that may be split,         */
                                 /* notch included; <= 0 means n_tets                  */
    void*          stream;       /* cudaStream_t for all device work (0 = legacy)      */
    int32_t        device;       /* CUDA device ordinal                                */
    cem_alloc_fn   alloc;        /* NULL: cudaMalloc                                   */
    cem_free_fn    free;         /* NULL: cudaFree                                     */
    void*          alloc_user;   /* passed to alloc/free                               */
    int64_t        n_instances;  /* <= 1: one specimen.  > 1: the mesh is a disjoint   */
                                 /* union of independent specimens (an ensemble)       */
    const int32_t* tet_instance; /* T specimen ids in [0, n_instances) (NULL if <= 1); */
                                 /* the elements of one specimen share no node with    */
                                 /* another's; each specimen gets its own time step    */
    int32_t        split_mode;   /* CEM_SPLIT_SUBDIVIDE (0) or CEM_SPLIT_DEACTIVATE;    */
                                 /* applies to the notch as well                       */
    int32_t        g_variant;    /* CEM_G_PRINCIPAL (0) or CEM_G_NORMAL                 */
    int64_t        n_dirichlet;  /* D >= 0 prescribed velocity components (Sec. 4.1-  */
                                 /* 4.3, 4.5): component dir_comp[q] of node           */
                                 /* dir_node[q] follows v(t) = min(t / t0, 1) dir_v0[q]*/
                                 /* with a = dir_v0[q] / t0 while t < t0, else 0.  The */
                                 /* values overwrite the corrector's v and a at the end*/
                                 /* of every step and at t = 0; nodes created by splits*/
                                 /* are free.  (node, component) pairs are distinct.   */
    const int32_t* dir_node;     /* D input node ids                                   */
    const uint8_t* dir_comp;     /* D components in {0, 1, 2}                          */
    const double*  dir_v0;       /* D final velocities [m/s]                           */
    double         dir_t0;       /* ramp time t0 [s]; <= 0: v = v0 from t = 0          */
    int32_t        elem_type;    /* CEM_ELEM_TET4 (0) or CEM_ELEM_HEX8.  HEX8: `tets`   */
                                 /* holds n_tets x 8 node ids (local order: the face   */
                                 /* z- counter-clockwise seen from z+, then the face   */
                                 /* z+ in the same order; positive volume required),   */
                                 /* split_enabled and n_notch must be 0, one specimen. */
                                 /* Smoothing domains take 1/12 of each hexahedron of  */
                                 /* an edge's fan; element strains are sampled at the  */
                                 /* edge midpoints with mean-corrected gradients.      */
    int32_t        tface_nodes;  /* nodes per traction face: 3 (or 0: triangles, load  */
                                 /* t A / 3 per node) or 4 (bilinear quadrilaterals,   */
                                 /* load t * integral of N_a dA)                       */
} cem_mesh_desc;

typedef struct cem_ctx cem_ctx;

/* Energies of the current state (Sec. 2.1, Eq. 2 terms). */
typedef struct cem_energy_t {
    double  kinetic;     /* 1/2 sum_i m_i |v_i|^2                                       */
    double  strain;      /* sum_k 1/2 Vs_k eps_k . sigma_k (smoothed edge strains)       */
    double  ext_work;    /* f_ext . u (load held constant)                               */
    double  dissipated;  /* U_d = sum over runtime splits of Gc * crack area            */
    double  modified;    /* kinetic + strain - ext_work - dt^2/8 a.M.a, conserved by    */
                         /* the central-difference map while the topology is fixed     */
    int64_t step;        /* completed steps                                             */
    double  time;        /* step * dt [s]                                               */
    int64_t n_split;     /* elements split at run time (notch excluded)                 */
} cem_energy_t;

/* Sizes and the time step of a context. */
typedef struct cem_info_t {
    int64_t n_nodes;         /* current nodes (input + split nodes)                     */
    int64_t n_tets;          /* current element slots (input + sub-elements)            */
    int64_t n_active_tets;   /* elements taking part in the step                        */
    int64_t n_edges;         /* current edges (smoothing domains)                       */
    int64_t n_candidates;    /* current crack-front elements                            */
    int64_t n_orig_edges;    /* edges of the input mesh                                 */
    double  dt;              /* time step [s]                                           */
    double  h_min;           /* min over input elements of 3V / max face area [m]       */
    int64_t device_bytes;    /* device memory held by the context                       */
    int64_t n_reorder;       /* node renumberings so far (cem_set_reorder)              */
    int64_t persistent_blocks; /* blocks of the last cem_step_persistent launch (0: none)  */
} cem_info_t;

/* Build the device mesh: edges and their element fans (Sec. 2.2, Fig. 4),
 * node incidence, face adjacency, traction load, prescribed velocities, and
 * apply the notch splits with the same rule as run-time splits.  Errors:
 * CEM_EINVAL (counts, ids out of range, zero-volume element, bad side mask,
 * unknown split_mode or g_variant, a repeated or out-of-range prescribed
 * component), CEM_ENOMEM, CEM_ECUDA.
 * On success *out owns all device memory of the context. */
int cem_mesh_create(const cem_mesh_desc* d, cem_ctx** out);

/* Material (Sec. 2.1): density rho [kg/m^3], Poisson ratio nu, Young's
 * modulus E [Pa] (nE = 1: uniform, nE = n_tets: per input element) and
 * critical energy release rate Gc [J/m^2] (nGc = 1 or n_tets).  Computes the
 * Lame constants, fan-averaged elasticity, lumped mass (Eq. 11), the time
 * step when automatic (per specimen of an ensemble, from its own elements),
 * and a_0 = M^-1 (f_ext - f_int(0)).  Required before
 * the first cem_step; CEM_ESTATE afterwards. */
int cem_set_material(cem_ctx* ctx, double rho, double nu,
                     const double* E, int64_t nE, const double* Gc, int64_t nGc);

/* Advance n >= 0 explicit steps (Eqs. 13-15, beta = 0, gamma = 1/2).  After
 * each step the energy release rates G_I, G_II (Eqs. 16-18) of every
 * crack-front element are evaluated on the end-of-step state, and every
 * element with max(G_I, G_II) > Gc is split (Sec. 3).  While crack-front
 * elements exist, the steps are launched in batches and the host reads the
 * split decision once per batch (see cem_set_step_batch); the results are
 * those of one step at a time, bit for bit.  Errors: CEM_ESTATE (no
 * material); CEM_ECAPACITY: when the split capacity would be exceeded the
 * splits of that step are not applied and the state is the step's
 * end-of-step kinematics (the context stays usable); when a storage
 * capacity (new edges, nodes, fan or incidence pool) runs out while splits
 * are applied, the step's topology is partly updated and the context should
 * be destroyed; CEM_ETIMEOUT (a bounded device wait gave up; as the second
 * ECAPACITY case); CEM_ENONFINITE (a displacement became non-finite);
 * CEM_ECUDA. */
int cem_step(cem_ctx* ctx, int64_t n);

/* Longest step batch of cem_step (no counterpart in the paper).  While
 * crack-front elements exist, cem_step launches up to max_steps steps back to
 * back.  The front evaluation of each step leaves its split decision on the
 * device; when one decides splits, the kernels of the batch's later steps
 * return at once without touching the state, the host applies the splits
 * after that step and continues from there.  A batch's length doubles after
 * every batch without a split, up to max_steps, and restarts at 1 after a
 * split.  max_steps = 1 reads the decision after every step.  Default 32.
 * Errors: CEM_EINVAL (max_steps < 1). */
int cem_set_step_batch(cem_ctx* ctx, int64_t max_steps);

/* The same n steps as cem_step, launched as one CUDA graph (no counterpart in
 * the paper).  Without crack-front elements (splitting disabled with
 * split_enabled = 0, the notch still applied at creation, or none left) the
 * graph holds the n steps.  With them it holds one batch of n steps as
 * cem_set_step_batch describes: when a step's front evaluation decides
 * splits, the graph's later steps return at once, the host applies the
 * splits, and the rest of the n steps run as cem_step runs them (the
 * topology changed, so that part is not replayed).  While the crack is
 * active (a step split and no step since has run without a split) the call
 * runs as cem_step does, without a capture, since a replay would end at its
 * first step.  The graph is captured on
 * a private stream on the first call and re-captured when n, the mesh sizes,
 * the crack-front count, the topology or the launch variants change; later
 * calls replay it on the context's stream.  Results are bit-identical to
 * cem_step.  Synchronises once at the end (to read the split decision and
 * check for non-finite displacements).  Errors: CEM_ESTATE (no material;
 * prescribed velocities, whose values depend on the step number; kernel
 * timing on), CEM_ENONFINITE, CEM_ETIMEOUT, CEM_ECAPACITY (as cem_step),
 * CEM_ECUDA. */
int cem_step_graph(cem_ctx* ctx, int64_t n);

/* The same n steps as cem_step, for a fixed topology, in one persistent
 * cooperative kernel launch (no counterpart in the paper).  The kernel's
 * 64-thread blocks are all resident at once (as many as the largest phase has
 * items for, at most the device's co-resident count); each phase of a step
 * (strain, edge stress, force, node update with the next step's predictor)
 * strides over its elements, edges or nodes, and a grid barrier separates the
 * phases, so a step costs four barriers instead of four or five kernel
 * launches.  That pays on small and medium meshes; on large ones the tuned
 * kernels of cem_step are faster.  Results are bit-identical to cem_step.  Valid while no step
 * can split (splitting disabled, or no crack-front element), tetrahedral
 * meshes only.  The barrier waits are bounded (cem_set_wait_limit): a wait
 * that gives up ends the launch and the call returns CEM_ETIMEOUT; the step
 * counter then stays where it was, but the node state is partly advanced (not
 * that of any step) and should be restored from a checkpoint.  Synchronises
 * once at the end.  Errors: CEM_ESTATE (no material; a hexahedral mesh;
 * crack-front elements with splitting on; prescribed velocities; kernel
 * timing on; no cooperative launch on the device), CEM_ETIMEOUT,
 * CEM_ENONFINITE, CEM_ECUDA. */
int cem_step_persistent(cem_ctx* ctx, int64_t n);

/* Bounded device waits.  Every spin-wait in the library's kernels (the
 * look-back of the ordered scans) gives up after a number of polls, records
 * an error flag and returns; the host then reports CEM_ETIMEOUT instead of
 * hanging.  cem_set_wait_limit sets that number (spins > 0; 0 restores the
 * default of 4,194,304 polls, about a second).  cem_wait_probe runs one
 * bounded wait on a device flag that nothing sets, as a check of this path:
 * it returns CEM_ETIMEOUT after the limit and leaves the context usable.
 * Neither has a counterpart in the paper. */
int cem_set_wait_limit(cem_ctx* ctx, int64_t spins);
int cem_wait_probe(cem_ctx* ctx);

/* Discrete adjoint of n_steps explicit steps from the current state, with the
 * topology fixed (requires split_enabled = 0; one specimen).  Objective
 *   J = c_strain * 1/2 u_N^T K u_N + sum_i w_u[i] . u_N[i]
 * (w_u: host, n_nodes x 3 row-major, or NULL).  Returns J, dJ_dE (host,
 * n_tets input elements; a split element's sub-elements add to it) and
 * dJ_dalpha, the derivative with respect to the traction amplitude alpha in
 * f_ext = alpha f_ext at alpha = 1 (a call from step 0 includes the
 * dependence of a_0 on alpha).  The adjoint of Eqs. 13-15 is not in the
 * paper.  States are kept every checkpoint_every steps (<= 0: ceil(sqrt(n)))
 * and each segment is recomputed before its reverse sweep.  The context ends
 * at step + n_steps.  Allocates its working memory through the context's
 * allocator and frees it before returning.  Errors: CEM_ESTATE (no material,
 * splitting on, ensemble, prescribed velocities), CEM_ENOMEM, CEM_ECUDA. */
int cem_adjoint(cem_ctx* ctx, int64_t n_steps, int64_t checkpoint_every, double c_strain,
                const double* w_u, double* J, double* dJ_dE, double* dJ_dalpha);

/* Energies of the current state (deterministic reductions). */
int cem_energy(cem_ctx* ctx, cem_energy_t* out);

/* Energies of one specimen of an ensemble (instance in [0, n_instances); 0
 * for a single specimen).  `time` is step * that specimen's time step. */
int cem_energy_instance(cem_ctx* ctx, int64_t instance, cem_energy_t* out);

/* Split original elements sorted by (step, element id).  The notch elements
 * appear with step = -1 and G = 0.  Writes min(count, cap) records to the
 * (optional, may be NULL) arrays and the total count to *n_split. */
int cem_crack_state(cem_ctx* ctx, int64_t* n_split, int32_t* tet, int8_t* pattern,
                    uint8_t* side, int64_t* step, double* G, int64_t cap);

/* Copy a node field (CEM_FIELD_*) as n_nodes x 3 row-major doubles into out
 * (capacity cap doubles; out may be NULL to query the size).  *n_nodes
 * receives the current node count. */
int cem_get_field(cem_ctx* ctx, int which, double* out, int64_t cap, int64_t* n_nodes);

/* Sizes and time step. */
int cem_info(cem_ctx* ctx, cem_info_t* out);

/* Kernel timing.  cem_profile(ctx, k) with k >= 1 clears the counters and
 * starts recording a pair of CUDA events (on the context's stream) around
 * the hot-path kernels below on every k-th step (events between kernels stop
 * a kernel's launch from overlapping the previous one, so sampling keeps the
 * other steps undisturbed); cem_profile(ctx, 0) stops.
 * cem_profile_read copies, for the first n kernel classes, the summed device
 * time in milliseconds and the number of timed launches (either array may be
 * NULL) and, in *total_launches (may be NULL), the number of kernels of any
 * kind the context launched since the last cem_profile(ctx, k >= 1).  Timing adds
 * two event records per launch; it does not change results. */
#define CEM_KERNEL_PREDICT     0   /* u <- u + dt v + dt^2/2 a (FP64 path; in mixed */
                                   /* precision the node update carries it)         */
#define CEM_KERNEL_STRAIN      1   /* per-element V * strain                        */
#define CEM_KERNEL_EDGE_STRESS 2   /* fan sum, smoothed edge stress                 */
#define CEM_KERNEL_FORCE       3   /* per-element nodal forces                      */
#define CEM_KERNEL_NODE_UPDATE 4   /* nodal force gather, acceleration, velocity    */
                                   /* (mixed: also u and the next predictor)        */
#define CEM_KERNEL_FRONT_G     5   /* energy release rates and split decisions      */
#define CEM_KERNEL_SPLIT       6   /* the whole split sequence of one step          */
#define CEM_KERNEL_COUNT       7
int cem_profile(cem_ctx* ctx, int enable);
int cem_profile_read(cem_ctx* ctx, double* ms, int64_t* launches, int n, int64_t* total_launches);

/* Autotuner of the step kernels' launch variants (no counterpart in the
 * paper).  Four kernels have variants: CEM_TUNE_STRAIN (per-element strain),
 * CEM_TUNE_EDGE (edge stress, a gather over each edge's element fan),
 * CEM_TUNE_FORCE (per-element forces) and CEM_TUNE_NODE (node update, a
 * gather over each node's element incidence).  A variant is a block size
 * (128, 256 or 512 threads) and, for the two gathers, how many list entries
 * have their loads issued together (fan: 2, 4 or 8, in edge order, or 102,
 * 104, 108 for 2, 4, 8 with each block's edges handed to its threads sorted by
 * fan size, so the edges of a warp have nearly equal fans, or 200 for the
 * block's strain records gathered into shared memory by TMA tile::gather4
 * copies, four records per copy, before the threads sum them; incidence: 2, 4
 * or 8, or 128 for warp-balanced rounds of up to 128 entries).  The TMA
 * variant's wait for its copies is bounded (cem_set_wait_limit): a wait that
 * gives up makes cem_step return CEM_ETIMEOUT.  cem_autotune does not time the
 * TMA variant (it measured slower than the others on GB300); cem_tune_set
 * selects it.
 * All variants of a kernel compute the same values in the same order: the
 * choice never changes results, only speed.
 *
 * cem_autotune times every variant on the context's current mesh and state
 * (CUDA events, one warm-up launch then `reps` launches; reps <= 0 means 5),
 * keeps the fastest, and records it under (GPU name, kernel, precision,
 * size bucket): floor(log2(item count)), floor(2 log2(node count)) for the
 * node update.  cache_path (may be NULL) names a text file that is read first
 * (entries found there are used without timing) and appended with new
 * results.  automatic != 0 makes cem_step re-tune a kernel (from the cache
 * when possible) whenever its item count (elements, edges or nodes) enters a
 * new bucket.  The state of the simulation is
 * unchanged.  The first call allocates one 3 x (node capacity) double buffer
 * through the context's allocator, held until cem_destroy.  Errors:
 * CEM_ESTATE (no material), CEM_EINVAL, CEM_ENOMEM, CEM_ECUDA.
 *
 * cem_tune_get reports kernel k's current variant and, from its last tuning,
 * the time per launch of that variant and of the untuned default (us; 0 if
 * the kernel was never timed, e.g. taken from the cache).  Any output
 * pointer may be NULL. */
#define CEM_TUNE_STRAIN 0
#define CEM_TUNE_EDGE   1
#define CEM_TUNE_FORCE  2
#define CEM_TUNE_NODE   3
#define CEM_TUNE_COUNT  4
int cem_autotune(cem_ctx* ctx, const char* cache_path, int reps, int automatic);
int cem_tune_get(cem_ctx* ctx, int kernel, int* block, int* batch, double* us, double* default_us);
/* Pin kernel k's variant (block in {128, 256, 512}; batch 1 for strain and
 * force, {2, 4, 8, 102, 104, 108, 200} for the edge stress, {2, 4, 8, 128} for
 * the node update,
 * where 128 selects warp-balanced gathers in rounds of 128 entries).  An
 * automatic autotuner may replace it when the kernel's bucket changes.
 * CEM_EINVAL for an unknown kernel or variant. */
int cem_tune_set(cem_ctx* ctx, int kernel, int block, int batch);

/* Diagnostics (no counterpart in the paper): measured FP64 FMA throughput of
 * `device` in FLOP/s (an FMA counts as two), timed with CUDA events on
 * `stream`.  The FP64 step kernels are bounded by this rate on GB300.
 * Allocates and frees a small device buffer itself. */
int cem_probe_fp64_fma(int device, void* stream, double* flops_per_s);

/* Diagnostics (no counterpart in the paper): the integer-only conversions of
 * the mixed-precision node update on the current device, for n host values:
 * (hi[i], lo[i]) = the FP32 pair of x[i] (x truncated to 24 significant bits,
 * then the remainder truncated to 24 bits; for |x| outside [2^-74, 2^128)
 * other than zero, the rounded pair RN(x), RN(x - RN(x))) and fd[i] = f[i] as
 * a double.  Synchronous; allocates and frees its own device buffers. */
int cem_probe_split(const double* x, const float* f, int64_t n, float* hi, float* lo, double* fd);

/* Diagnostics: the split rule of Sec. 3 (the sub-elements that replace a
 * split element, each remaining prism divided into three tetrahedra) run on
 * the current device with the device code cem_step uses, for n host cases.
 * Case q: nodes[4q..4q+3] the element's node indices, ids[4q..] their
 * creation ids, mask[q] its side mask (1..14: bit l = side of local node l),
 * mnode[16q + 4x + y] / mid[16q + 4x + y] the new node on local edge x-y that
 * stays attached to x, and its creation id.  Writes subs[24q + 4r + c] = node
 * c of sub-element r (r < count[q]; later rows -1) and count[q] (6 for
 * pattern I, 4 for pattern II), before orientation.  CEM_EINVAL for a null
 * pointer or a mask outside 1..14; synchronous; allocates and frees its own
 * device buffers. */
int cem_probe_split_rule(int64_t n, const int32_t* nodes, const int32_t* ids, const int32_t* mask,
                         const int32_t* mnode, const int32_t* mid, int32_t* subs, int32_t* count);

/* Nodal energy sums of caller-owned device arrays, with no allocation.  The
 * paper has no counterpart: this is a library facility for callers that
 * cannot call cudaMalloc, for example code whose device memory is entirely
 * reserved by another allocator (a caching allocator holding the free memory
 * makes a raw cudaMalloc fail) or code running under a fixed device-memory
 * budget.  It computes, into out[0..2] (device memory, written on `stream`):
 *   out[0] = 1/2 sum_i mass[i] |v_i|^2,  out[1] = sum_i f_ext_i . u_i,
 *   out[2] = sum_i mass[i] |a_i|^2,
 * the nodal terms of cem_energy.  u, v, a, fext are [3][ld] structure-of-
 * arrays device arrays (component c of node i at c*ld + i), mass is [n_nodes].
 * The block partial sums live in one fixed 96 KiB __device__ array per GPU
 * (held by every GPU that loads the library until the process exits), which
 * bounds n_nodes to 16,777,216: larger counts return CEM_ECAPACITY without
 * touching the GPU.  Bad pointers or ld < n_nodes return CEM_EINVAL.  The
 * first call on a device looks up that array's address (cudaGetSymbolAddress)
 * with the device current; make that first call before any stream capture
 * begins.  All calls on a device share the array: calls that overlap on the
 * GPU race and give wrong sums.  Calls no cudaMalloc, cudaFree or allocating
 * library routine.  An error already pending on the calling thread (from
 * earlier work) is reported as CEM_ECUDA and left pending, with nothing
 * launched. */
int cem_node_energies_noalloc(const double* u, const double* v, const double* a, const double* mass,
                              const double* fext, int64_t n_nodes, int64_t ld, double* out, void* stream);

/* Node renumbering for memory locality (no counterpart in the paper).  Split
 * nodes are appended to the node arrays, so an element made by a split pairs
 * nodes whose storage lies far apart, and the node update gathers its force
 * record from DRAM once per such node.  A renumbering puts the nodes in
 * Morton order of their reference coordinates (ties by id) and rewrites the
 * incidence lists in that order.  It changes only where nodes are stored:
 * every function of this header keeps taking and returning nodes by their
 * creation ids (input nodes first, then split nodes in the order they were
 * made), and every result is bit-identical to a run without renumbering
 * except for the last bits of energy sums, which add nodes in storage order.
 * cem_set_reorder sets the trigger: after a split step, renumber when the
 * node count has grown by the fraction `growth` since the last renumbering
 * (or since the input mesh); growth = 0 never renumbers.  Default 0.25 for
 * tetrahedral meshes with splitting; CEM_EINVAL for growth < 0.
 * cem_reorder_nodes renumbers now.  Both return CEM_ESTATE for contexts
 * without splitting (hexahedral or split_enabled = 0), whose node order is
 * the input's. */
int cem_set_reorder(cem_ctx* ctx, double growth);
int cem_reorder_nodes(cem_ctx* ctx);

/* Checkpoint and resume.  cem_save writes the context's dynamic state to the
 * file `path`: node, element and edge arrays up to their current counts, the
 * fan and incidence lists, the crack records, the candidate list, the
 * new-node and new-edge maps, U_d and the step counter (not the step's
 * scratch, which every step rewrites before reading).  cem_load reads such a
 * file into a context created from the same mesh description with the same
 * material; stepping it then continues bit for bit as the saved context
 * would have.  Both synchronise the context's stream and return after the
 * file is written / the state is on the device.  The file ends with a
 * 64-bit FNV-1a hash of its bytes; cem_load reads and checks the whole file
 * before it changes the context.  Errors: CEM_ESTATE (no material),
 * CEM_EINVAL (cannot open or write the file; not a checkpoint; a different
 * mesh, element type, precision, capacity or time step; a truncated or
 * corrupted file: in all of these the context is left as it was; a file
 * that changes while it is being loaded, after which the context's state is
 * undefined), CEM_ECUDA.  In the same first pass every index array is
 * range-checked (node, element, edge and pool indices within the file's
 * counts, every fan and incidence list inside its pool's used part, the node
 * storage order a permutation): a file with an index out of range returns
 * CEM_EINVAL and leaves the context as it was.  Floating-point contents are
 * not checked.  The file is in host byte order. */
int cem_save(cem_ctx* ctx, const char* path);
int cem_load(cem_ctx* ctx, const char* path);

/* Release every device allocation and the context (NULL is accepted). */
int cem_destroy(cem_ctx* ctx);

/* Message of the last error on ctx ("" when none).  With ctx == NULL: the message
 * of the last failed cem_mesh_create on this host thread. */
const char* cem_last_error(const cem_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* CEM_H */
