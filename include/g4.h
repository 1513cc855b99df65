/*
 * g4.h -- C ABI of the GB300 short-range tree / FMM gravity library (libg4.so).
 *
 * The library computes the short-range gravitational accelerations and potentials of the
 * GADGET-4 method (Springel, Pakmor, Zier & Reinecke 2021) on one GPU:
 *   integer coordinates (Sec. 2.10, 2.11) -> Peano-Hilbert keys and radix sort (Sec. 2.2.1)
 *   -> oct-tree with leaf threshold (Sec. 2.2.1) -> node moments (Sec. 2.2.2)
 *   -> one-sided tree walk with the relative opening criterion (Eq. eqnrelcriterion) and the
 *      TreePM short-range kernel (Eq. eqnpo4), or the symmetric Cartesian FMM (Sec. 2.4).
 *
 * Conventions for every entry point:
 *   - All array arguments are DEVICE pointers owned by the caller, unless stated otherwise.
 *     Only a g4_tree handle is library-owned (create with g4_tree_create, release with
 *     g4_tree_free).
 *   - Every call is asynchronous on `stream` (a cudaStream_t passed as void*; NULL = legacy
 *     default stream).  The returned status reports argument and launch errors synchronously.
 *     Errors detected by kernels (capacity overflow, bounded waits running out) are recorded
 *     in the tree handle and reported by g4_tree_status(), which synchronises the stream.
 *   - Integer positions are uint32 per axis in SoA layout [x[0..n), y[0..n), z[0..n)]; the
 *     physical unit of one integer step is box_size / 2^32 (Sec. 2.10).
 *   - Potential sign convention: pot = phi = -G sum m g(r); acc = -grad phi (Sec. 2.2.2).
 *     The constant pi/(alpha^2 V) of Eq. (eqnpo4) is omitted and the self-potential of a
 *     particle is not included.
 *   - On failure a thread-local message is available from g4_last_error().
 *   - The library never falls back to a CPU path: without a usable CUDA device every call
 *     that launches work returns G4_ERR_CUDA.
 */
#ifndef G4_H
#define G4_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    G4_OK = 0,
    G4_ERR_INVALID_ARG = 1, /* bad pointer, size or parameter */
    G4_ERR_OOM = 2,         /* device allocation failed */
    G4_ERR_CUDA = 3,        /* CUDA launch or runtime error */
    G4_ERR_TIMEOUT = 4,     /* a bounded device wait ran out */
    G4_ERR_DEPTH = 5,       /* key resolution exceeded */
    G4_ERR_STATE = 6,       /* handle used in the wrong order (e.g. walk before moments) */
    G4_ERR_CAPACITY = 7     /* a library-owned buffer was too small; retry with more */
} g4_status;

#define G4_MAX_EPS_CLASSES 8
#define G4_MAX_ORDER 5

/* Parameters of one force computation (plain values, copied by every call). */
typedef struct g4_params {
    double box_size;       /* L; physical size of the 2^32 integer range (Sec. 2.10) */
    int periodic;          /* 1: nearest periodic image via two's complement (Sec. 2.10) */
    double r_s;            /* TreePM split scale (Sec. 2.3); <= 0: plain Newtonian kernel */
    double r_cut_factor;   /* R_cut; r_cut = max(R_cut * r_s, 2.8 eps_max) (Sec. 2.3) */
    int pp_cut;            /* 1: particle pairs with r >= r_cut are dropped (TreePM only).
                              0: every pair of each leaf the walk reaches is kept; leaves
                              are skipped per group of sinks (conservatively), so that set
                              depends on the grouping: a diagnostic mode */
    double alpha;          /* relative opening parameter of Eq. (eqnrelcriterion) */
    double theta;          /* geometric opening angle theta_c (criterion 1, bootstrap) */
    int criterion;         /* 0: relative criterion (needs a_old), 1: geometric l/r < theta */
    int order_p;           /* expansion order p, 1..5 (Sec. 2.2.2) */
    int leaf_max;          /* split threshold: a node with more particles is split (1..64) */
    int exclusion_zone;    /* 1: no multipole use within the cube of half-width l around the
                              node's geometric centre (Sec. 2.2.3) */
    int precision;         /* 0: FP32 interactions, FP64 moments for big nodes; 1: all FP64 */
    double G;              /* gravitational constant */
    int n_eps_classes;     /* number of softening classes (1..G4_MAX_EPS_CLASSES) */
    double eps_table[G4_MAX_EPS_CLASSES]; /* softening length eps_0 per class (Sec. 2.7) */
    int group_size;        /* sinks per warp group of the tree walk: 8, 16 or 32 (0 = 32);
                              smaller groups stage fewer sources per sink but leave lanes
                              idle.  Forests, LPT orders and work items use 32. */
    int fp64_count;        /* nodes holding >= fp64_count particles accumulate moments in
                              FP64 (0 = 4096) */
    int keep_qp;           /* FMM: 1 keeps Q_p in the potential (Sec. 2.4 drops it) */
    int fmm_p2p_per_particle; /* FMM: deferred particle-pair list entries per particle of
                              the handle (0 = 16); beyond them the dual walk evaluates the
                              pairs itself */
    int soft_nodes;        /* 0: a particle-node pair (tree walk, FMM) or node-node pair (FMM)
                              closer than 2.8 eps_ij, eps_ij = the larger of the two sides'
                              largest softenings, is opened (GADGET-3, multipoles unsoftened);
                              1: the GADGET-4 rule of Sec. 2.7, such a pair is opened only if
                              both sides' smallest softenings lie below eps_ij (a particle's
                              smallest is its own), otherwise it interacts through the
                              expansion of the softened kernel with eps_ij */
    int ewald;             /* periodic=1 and r_s=0 only: 1 adds the Ewald correction psi of
                              Eq. (eqnewal) to every interaction -- the pure periodic tree and
                              FMM of Sec. 2.2.4: nearest-image Newtonian terms plus the
                              correction, expanded like them (tree: about each accepted node's
                              centre of mass; FMM: in every mutual expansion, the kernel
                              1/r - psi), for every particle pair, and G m_i psi(0) of each
                              particle's own images in its potential.  D_n[psi] come
                              from a grid of the tensors up to order p + 4 (one octant, 32^3
                              cells, FP64 from the Ewald sums, built in the handle on first
                              use) by third-order Taylor expansion about the nearest cell
                              centre.  0: nearest images only. */
    long long watchdog_cycles; /* tree walk work-queue watchdog: 0 none; > 0: a warp takes no
                              further work once it has run that many SM clock cycles, the
                              walk's results are then incomplete and g4_tree_status reports
                              G4_ERR_TIMEOUT (until the next g4_tree_build clears the flags).
                              A bounded run time for callers that must not wait on a
                              runaway walk; nothing spins, the kernel ends normally. */
} g4_params;

typedef struct g4_tree_s *g4_tree;

/* Library version string (static storage). */
const char *g4_version(void);

/* Thread-local description of the last error returned on this thread (static storage). */
const char *g4_last_error(void);

/* Number of kernel launches the library has issued since it was loaded (all threads).
 * Diagnostic only; host-side, never fails. */
int64_t g4_launch_count(void);

/* Fills *p with the defaults: periodic=0, r_s=0, R_cut=4.5, pp_cut=1, alpha=0.0025,
 * theta=0.5, criterion=0, p=3, leaf_max=8, exclusion=1, precision=0, G=1, one class with
 * eps=0.01, group_size=32, fp64_count=4096, keep_qp=0, fmm_p2p_per_particle=0, soft_nodes=0,
 * ewald=0, watchdog_cycles=0.
 * Host-only, never fails for p!=NULL. */
g4_status g4_params_default(g4_params *p);

/* ---- pure periodic tree: the Ewald correction grid (Sec. 2.2.4) ---------------------- */

/* Evaluates the derivative tensors D_abc[psi](x), a + b + c <= nmax (0..6), of the Ewald
 * correction potential for a cubic box of side `box` at n separations x[n][3] (FP64,
 * row-major, device, each component in [-box/2, box/2]: nearest-image separations), from the
 * handle's grid (built or rebuilt for `box` first, as the walk does) by third-order Taylor
 * expansion in FP64.  out: device, n x (nmax+1)(nmax+2)(nmax+3)/6 doubles, component
 * (a, b, c) of order m at (m(m+1)(m+2)/6 + (b+c)(b+c+1)/2 + c).  Asynchronous on `stream`;
 * errors: G4_ERR_INVALID_ARG, G4_ERR_OOM (grid allocation, first use only). */
g4_status g4_ewald_eval(g4_tree t, const double *x, int64_t n, int nmax, double box, double *out,
                        void *stream);

/* ---- a1: integer coordinates (Sec. 2.10, Sec. 2.11) ----------------------------------- */

/* Converts n physical positions pos[n][3] (FP64, row-major, device) to uint32 SoA
 * pos_int[3][n] (device).
 *   periodic = 1: x_int = floor(x / L * 2^32) mod 2^32, L = box_size; frame = {0,0,0,L}.
 *   periodic = 0: the bounding box is shrink-wrapped into the central half of the integer
 *     cube: S = smallest power of two >= 2 * (largest extent), centred on the bounding-box
 *     midpoint c: x_int = floor((x - c) * 2^32 / S) + 2^31; frame = {c - S/2 (3), S}
 *     (box_size is ignored).
 * frame: 8 doubles of device memory (caller-owned); receives {origin_x, origin_y, origin_z,
 * side} in its first four, the rest is the call's own scratch (the bounding-box reduction
 * runs in this buffer, so the call allocates nothing, never synchronises, and calls with
 * different frame buffers may overlap).  The isolated case needs `side` as params.box_size
 * of the later calls.
 * Errors: G4_ERR_INVALID_ARG for NULL pointers, n < 0 or box_size <= 0 when periodic. */
g4_status g4_int_coords(const double *pos, int64_t n, int periodic, double box_size,
                        uint32_t *pos_int, double *frame, void *stream);

/* ---- a2 + a3: Peano-Hilbert keys and stable radix sort (Sec. 2.2.1) -------------------- */

/* Bytes of device workspace g4_keys_sort needs for n particles. */
g4_status g4_keys_sort_workspace(int64_t n, size_t *bytes);

/* 63-bit Peano-Hilbert keys from the top 21 bits of each coordinate, then a stable sort:
 *   keys_sorted[k] = key of particle perm[k], ascending; equal keys keep input order.
 * pos_int: 3 x n SoA (device); keys_sorted: n uint64 (device); perm: n int32 (device,
 * sorted -> original index).  workspace: >= g4_keys_sort_workspace(n) bytes of device
 * memory, 256-byte aligned, not used concurrently by another call.
 * Errors: G4_ERR_INVALID_ARG for NULL pointers, n < 0, n >= 2^31, small workspace. */
g4_status g4_keys_sort(const uint32_t *pos_int, int64_t n, uint64_t *keys_sorted,
                       int32_t *perm, void *workspace, size_t workspace_bytes, void *stream);

/* Same result as g4_keys_sort, but allocation-free: the scratch memory is a fixed array inside
 * the library (about 16 MB of device memory on every GPU that loads libg4, held until the
 * process exits) instead of a caller workspace.  The paper has no counterpart; this entry
 * point exists for callers that cannot allocate device memory when they sort -- applications
 * whose device memory belongs to another allocator, plugins handed pointers but no
 * allocator.  It calls no cudaMalloc/cudaFree.
 *   - n is limited to 2^20 (1048576); larger n returns G4_ERR_INVALID_ARG with a message.
 *   - The first call on a device looks up the array's device address (cudaGetSymbolAddress,
 *     with that device current) and caches it.
 *   - All calls share the array: calls that overlap on the GPU (other streams or threads)
 *     race on it and must be serialised.  Each call overwrites every scratch word it reads,
 *     so nothing needs clearing between calls.
 * Arguments and output as for g4_keys_sort. */
g4_status g4_keys_sort_noalloc(const uint32_t *pos_int, int64_t n, uint64_t *keys_sorted,
                               int32_t *perm, void *stream);

/* Batched independent systems (a forest), e.g. many small isolated systems solved together:
 * bytes of workspace for g4_keys_sort_batched. */
g4_status g4_keys_sort_batched_workspace(int64_t n, size_t *bytes);

/* Stable sort of n particles by (system id, Peano-Hilbert key): particles of system s end up
 * contiguous, in PH order within the system.  sys_id: n uint16 (device, < 65536 systems);
 * pos_int as for g4_keys_sort (each system in its own integer frame); keys_sorted, perm as
 * for g4_keys_sort; workspace >= g4_keys_sort_batched_workspace(n), 256-byte aligned. */
g4_status g4_keys_sort_batched(const uint32_t *pos_int, int64_t n, const uint16_t *sys_id,
                               uint64_t *keys_sorted, int32_t *perm, void *workspace,
                               size_t workspace_bytes, void *stream);

/* Gathers particle arrays into PH order: out[k] = in[perm[k]].  cls/aold may be NULL (both
 * in and out).  pos arrays are 3 x n SoA. */
g4_status g4_gather(const int32_t *perm, int64_t n, const uint32_t *pos_in,
                    const float *mass_in, const uint8_t *cls_in, const float *aold_in,
                    uint32_t *pos_out, float *mass_out, uint8_t *cls_out, float *aold_out,
                    void *stream);

/* Scatters PH-ordered results back to input order: out[perm[k]] = in[k].  acc arrays are
 * 3 x n SoA; pot may be NULL (both). */
g4_status g4_scatter(const int32_t *perm, int64_t n, const float *acc_sorted,
                     const float *pot_sorted, float *acc_out, float *pot_out, void *stream);

/* Active subsets (hierarchical time bins, where each force call builds its tree over the
 * active particles only): out[k] = in[idx[k]] for k < n_sub, where the input arrays hold
 * n_all particles (pos_in 3 x n_all SoA) and the outputs n_sub (pos_out 3 x n_sub SoA).
 * cls/aold may be NULL (both in and out). */
g4_status g4_gather_subset(const int32_t *idx, int64_t n_sub, int64_t n_all, const uint32_t *pos_in,
                           const float *mass_in, const uint8_t *cls_in, const float *aold_in,
                           uint32_t *pos_out, float *mass_out, uint8_t *cls_out, float *aold_out,
                           void *stream);

/* The inverse: acc_out[idx[k]] = acc_sub[k] (3 x n_sub into 3 x n_all SoA), pot likewise
 * (both NULL or both set). */
g4_status g4_scatter_subset(const int32_t *idx, int64_t n_sub, int64_t n_all, const float *acc_sub,
                            const float *pot_sub, float *acc_out, float *pot_out, void *stream);

/* ---- a4: oct-tree (Sec. 2.2.1) ---------------------------------------------------------- */

/* Allocates a tree handle for up to n_max particles and node_capacity nodes (0 = a default
 * that suffices for ordinary particle sets).  All device memory is allocated here, none in
 * later calls, so build/moments/walk sequences can be captured in a CUDA graph.
 * Errors: G4_ERR_INVALID_ARG, G4_ERR_OOM. */
g4_status g4_tree_create(int64_t n_max, int64_t node_capacity, g4_tree *out);

/* Releases the handle and its device memory (synchronises the device first). */
void g4_tree_free(g4_tree tree);

/* Builds the oct-tree over PH-sorted keys: a node is split when it holds more than
 * leaf_max particles and lies above the 21-level key resolution; children are in PH order;
 * nodes are numbered in depth-first pre-order.  pos_sorted (3 x n SoA, PH order) gives the
 * node cells.  Requires n <= n_max of the handle.  Capacity overflow is reported by
 * g4_tree_status (G4_ERR_CAPACITY). */
g4_status g4_tree_build(g4_tree tree, const uint64_t *keys_sorted, const uint32_t *pos_sorted,
                        int64_t n, const g4_params *params, void *stream);

/* Builds one oct-tree per system in a single call sequence (a forest; Sec. 2.2.1 per system).
 * keys_sorted/pos_sorted: output of g4_keys_sort_batched plus g4_gather; sys_first: n_sys + 1
 * int32 (device) giving each system's first sorted index (sys_first[n_sys] = n; systems must
 * be non-empty); sys_box: n_sys doubles (device), the physical size of each system's 2^32
 * integer range (the `side` of its isolated frame, or its periodic box).  Both arrays are
 * read by later g4_multipoles / g4_gravity_tree calls on this handle and must stay valid.
 * Roots are numbered in system order; g4_gravity_tree then walks each sink only through its
 * own system's tree, all systems in one persistent launch (params.box_size is ignored). */
g4_status g4_tree_build_forest(g4_tree tree, const uint64_t *keys_sorted,
                               const uint32_t *pos_sorted, int64_t n, const int32_t *sys_first,
                               const double *sys_box, int32_t n_sys, const g4_params *params,
                               void *stream);

/* Synchronises `stream`, then reports the node count, deepest level and the device error
 * flags of the last build/walk.  Returns G4_ERR_CAPACITY / G4_ERR_TIMEOUT when a kernel
 * recorded that condition (flags are cleared by the next g4_tree_build). */
g4_status g4_tree_status(g4_tree tree, int64_t *n_nodes, int32_t *max_level, void *stream);

/* Copies the node topology (depth-first order) into caller device buffers of at least
 * n_nodes entries: level, first particle, particle count, next (index after the subtree),
 * centre (n_nodes x 3 uint32, geometric centre in integer units).  Any pointer may be NULL. */
g4_status g4_tree_nodes(g4_tree tree, int32_t *level, int32_t *first, int32_t *count,
                        int32_t *next, uint32_t *center, void *stream);

/* ---- a5: node moments (Sec. 2.2.2) ------------------------------------------------------ */

/* Mass M, centre of mass s, multipole moments Q_2..Q_p about s (Q_1 = 0), per-node maximum
 * softening and minimum |a_old| (FMM).  Inputs in PH order; cls and aold may be NULL (class
 * 0 / |a| = 0).  Nodes with >= fp64_count particles accumulate in FP64. */
g4_status g4_multipoles(g4_tree tree, const uint32_t *pos_sorted, const float *mass_sorted,
                        const uint8_t *cls_sorted, const float *aold_sorted,
                        const g4_params *params, void *stream);

/* Copies node moments into caller device buffers (n_nodes entries each): mass, com
 * (n_nodes x 3, s minus geometric centre, physical units), mono (n_nodes x nmono, monomial
 * moments sum m dx^a dy^b dz^c of orders 0..p about s, multi-indices ordered by order, then
 * a descending, then b descending).  Any pointer may be NULL. */
g4_status g4_tree_moments(g4_tree tree, double *mass, double *com, double *mono, void *stream);

/* ---- a6/a7: one-sided tree walk (Sec. 2.2.3, Sec. 2.3) ---------------------------------- */

/* Accelerations and potentials of the sinks from all particles of the tree.
 *   sinks: active == NULL -> all n particles; otherwise active[0..n_active) lists sorted-order
 *          indices (ascending PH order recommended for coherent groups).
 *   opening: relative criterion G M / r^2 (l/r)^p < alpha |a_old| (criterion 0; aold_sorted
 *          required) or geometric l/r < theta (criterion 1); plus the exclusion zone, and
 *          nodes closer than 2.8 max(eps_i, eps_max(node)) are always opened.
 *   TreePM (r_s > 0): nodes whose nearest (periodic-image) edge is beyond r_cut are dropped;
 *          pairs use g = g_soft - erf(r / 2 r_s) / r (Eq. eqnpo4).
 * Outputs (sorted order, written only at sink indices): acc 3 x n SoA float, pot n float
 * (nullable), counts 2 x n uint32 (PP interactions, PN interactions; nullable).
 * Work: 32-sink groups from a device counter (persistent kernel), optionally in the order set
 * by g4_tree_set_group_order or as the parts set by g4_tree_set_work_items.  The handle keeps
 * walk copies (allocated on its first walk, outside any graph capture): the node records in
 * level order (rebuilt after each g4_multipoles) and 16-byte particle records (rewritten by
 * every call), plus per-warp frontier rings (a frontier overflow sets the list-capacity flag).
 * FP32 TreePM pairs use erfc(x) = exp(-x^2) erfcx(x) with a fitted erfcx (relative error
 * below 5e-7).  Requires g4_tree_build and g4_multipoles on the same handle with the same
 * order_p. */
g4_status g4_gravity_tree(g4_tree tree, const uint32_t *pos_sorted, const float *mass_sorted,
                          const uint8_t *cls_sorted, const float *aold_sorted,
                          const int32_t *active, int64_t n_active, const g4_params *params,
                          float *acc, float *pot, uint32_t *counts, void *stream);

/* g4_gravity_tree with the scatter back to input order fused into the walk's epilogue:
 * perm (n int32, device; g4_keys_sort's permutation, perm[s] = input index of sorted particle
 * s, a permutation of 0..n-1) sends sorted sink s's acceleration and potential to
 * acc[:, perm[s]] and pot[perm[s]] (acc 3 x n SoA and pot n in input order); counts stay in
 * sorted order.  Same results as g4_gravity_tree
 * followed by g4_scatter, without the sorted-order copies.  Errors: those of
 * g4_gravity_tree; G4_ERR_INVALID_ARG for a NULL perm. */
g4_status g4_gravity_tree_perm(g4_tree tree, const uint32_t *pos_sorted, const float *mass_sorted,
                               const uint8_t *cls_sorted, const float *aold_sorted,
                               const int32_t *active, int64_t n_active, const g4_params *params,
                               const int32_t *perm, float *acc, float *pot, uint32_t *counts,
                               void *stream);

/* ---- a8: symmetric Cartesian FMM (Sec. 2.4, Sec. 2.5) ----------------------------------- */

/* Bytes of device workspace g4_gravity_fmm needs, sized from the handle's node capacity and
 * n_max (no host synchronisation): field tensors, pass-down lists and the deferred
 * particle-pair lists (16 entries per particle plus a floor). */
g4_status g4_fmm_workspace(g4_tree tree, const g4_params *params, size_t *bytes);

/* Forces for all n particles by the dual tree walk over pairs of cells, a cell being a node or
 * a single particle (Sec. 2.4: a pair's members are nodes or single particles; a particle is a
 * cell of side 0 with Q_0 = m).  A pair interacts by the symmetric expansion (fields added to both
 * cells; at a particle the field is evaluated on the spot), or fails and is opened: both cells
 * ("open both"), a leaf into its particles, a particle never; two particles interact directly
 * (pair kernel).  A node paired with itself is replaced by all pairs of its daughters.
 * Criterion G M_max / r^2 (l_max/r)^(p-1) < alpha min |a|_min (a particle contributes its own
 * mass, side 0 and |a_old|), or (l_A + l_B)/r < theta; with the exclusion zone no pair
 * interacts whose centre separation is within max(l_A, l_B) along every axis (touching nodes,
 * a particle inside a node's exclusion cube); pairs closer than 2.8 max(eps) are opened;
 * pairs whose nearest faces are beyond r_cut are dropped.  Node fields are passed down (L2L)
 * and evaluated at the particles (L2P).  Particle pairs are recorded during the dual walk and
 * evaluated afterwards by a separate kernel with the tree walk's particle-particle phase
 * (when the workspace's lists are full, the dual walk evaluates them itself: same
 * interactions, possibly other rounding order).
 *   aold_sorted: |a_old| per sorted particle (required by the relative criterion; may be NULL
 *          for the geometric one).  The nodes' |a|_min come from g4_multipoles.
 *   counts: 3 x n uint32 (nullable): particle pairs of the particle, particle-node terms
 *          evaluated at the particle, node-node fields reaching its leaf.
 *   momentum_out: 3 doubles of device memory (nullable), receives sum m a in FP64.
 *   precision 1 (order_p 4 only; needs g4_multipoles with precision 1): the FP64 reference
 *          mode -- the decisions as in FP32, every expansion, field, downward shift and
 *          particle pair in FP64 from the FP64 node data; outputs still float.  Other orders:
 *          G4_ERR_INVALID_ARG; FP32 multipoles: G4_ERR_STATE.
 * Outputs otherwise as for g4_gravity_tree. */
g4_status g4_gravity_fmm(g4_tree tree, const uint32_t *pos_sorted, const float *mass_sorted,
                         const uint8_t *cls_sorted, const float *aold_sorted,
                         const g4_params *params, float *acc, float *pot, uint32_t *counts,
                         double *momentum_out, void *workspace, size_t workspace_bytes,
                         void *stream);

/* ---- long-range particle-mesh force of the TreePM split (Sec. 2.3) ------------------------ */

/* Bytes of device workspace g4_pm_long_range needs for an n_grid^3 mesh (n_grid a power of two
 * in [16, 1024]): a complex FP32 mesh (8 n_grid^3 bytes) and the FFT twiddles. */
g4_status g4_pm_workspace(int32_t n_grid, size_t *bytes);

/* Long-range accelerations and potentials of the TreePM split (Sec. 2.3: the Fourier sum of
 * Eq. eqnksum, with the sign that makes it add to the short-range part of Eq. eqnpo4 to give
 * the periodic potential of Eq. eqnpo1), by the particle-mesh steps the paper lists:
 *   clouds-in-cell assignment of the n sources to a periodic n_grid^3 mesh (mesh points at
 *   i * L / n_grid); FFT; multiplication with -4 pi G exp(-k^2 r_s^2) / k^2 divided by the
 *   CIC assignment and interpolation transforms, prod_i sinc^4(k_i Delta / 2) (Delta =
 *   L / n_grid); inverse FFT; fourth-order differences of the potential; CIC interpolation
 *   to the n_sinks sink positions.
 *   pos: sources, 3 x n uint32 SoA (integer coordinates, unit box_size / 2^32); mass: n floats;
 *   pos_sinks: 3 x n_sinks uint32 SoA (may be pos itself with n_sinks = n);
 *   params: box_size (L), periodic (must be 1), r_s (> 0), G;
 *   acc: 3 x n_sinks float SoA, pot: n_sinks floats (nullable); accumulate = 1 adds to them
 *   (e.g. to the tree's short-range forces of the same sinks), 0 overwrites.
 *   workspace: >= g4_pm_workspace(n_grid) bytes of device memory, 256-byte aligned.
 * The mesh sums use FP32 atomics, so results are reproducible to rounding, not bitwise.
 * Errors: G4_ERR_INVALID_ARG for a non-periodic box, r_s <= 0, a bad n_grid or workspace. */
g4_status g4_pm_long_range(const uint32_t *pos, const float *mass, int64_t n,
                           const uint32_t *pos_sinks, int64_t n_sinks, const g4_params *params,
                           int32_t n_grid, float *acc, float *pot, int accumulate,
                           void *workspace, size_t workspace_bytes, void *stream);

/* ---- hierarchical time integration (Sec. 4.2) --------------------------------------------- */

/* Kick operator K: vel[i] += dt * acc[i] for the particles listed in idx (n_idx sorted or
 * unsorted indices; idx = NULL: all n).  vel, acc: 3 x n float SoA (device). */
g4_status g4_kick(float *vel, const float *acc, const int32_t *idx, int64_t n_idx, int64_t n,
                  double dt, void *stream);

/* Drift operator D: pos[i] += rint(vel[i] * dt * 2^32 / box_size) for the listed particles, on
 * the integer coordinates (3 x n uint32 SoA): positions stay exact integers and a periodic box
 * wraps through the 32-bit overflow (Sec. 2.10).  For an isolated set (periodic = 0) a step that
 * would leave the central half of the integer cube is not applied and sets *flag (1 int32 of
 * device memory, required then) to 1. */
g4_status g4_drift(uint32_t *pos, const float *vel, const int32_t *idx, int64_t n_idx, int64_t n,
                   double dt, const g4_params *params, int32_t *flag, void *stream);

/* Timestep bins: dt_i = sqrt(2 eta eps_i / |a_i|) (eps_i from the particle's softening class,
 * cls NULL = class 0), bins[i] = the smallest k <= max_bin with dt_max / 2^k <= dt_i (0 for
 * |a_i| = 0): the power-of-two hierarchy in which the hierarchical scheme splits a system into
 * slow and fast particles.  acc 3 x n float, bins n uint8 (written at the listed indices). */
g4_status g4_timestep_bins(const float *acc, const uint8_t *cls, const int32_t *idx, int64_t n_idx,
                           int64_t n, const g4_params *params, double eta, double dt_max,
                           int32_t max_bin, uint8_t *bins, void *stream);

/* Random translation (Sec. 3.8): pos_out = pos_in + shift modulo 2^32 per axis, for n
 * particles (3 x n uint32 SoA, device; pos_out may equal pos_in).  shift: 3 uint32 in HOST
 * memory, read during the call.  With integer coordinates the shift is loss-less and exactly
 * reversible (add 2^32 - shift); in a periodic box it moves the particle set relative to the
 * root node, which decorrelates the tree's and the mesh's force errors between steps. */
g4_status g4_translate(const uint32_t *pos_in, uint32_t *pos_out, int64_t n, const uint32_t *shift,
                       void *stream);

/* ---- learned cost model for scheduling the walk (no counterpart in the paper's method; its
 *      load-balancing cost q_i is the interaction count of the last force computation,
 *      Sec. 6.1, which these calls learn to predict) --------------------------------------- */

/* Number of float parameters of the 6 -> 32 -> 32 -> 1 MLP (1313): W1[32][6], b1[32],
 * W2[32][32], b2[32], W3[32], b3. */
int32_t g4_mlp_param_count(void);

/* Six features per PH-sorted particle of a built tree, row-major n x 6 floats: leaf
 * occupancy / leaf_max, leaf depth / 21, log10 |a_old|, time bin / 8, log2(parent count)/24,
 * log2(grandparent count)/24.  aold_sorted, bins_sorted (uint8 time bins) may be NULL.
 * leaf_scratch: n int32 of device scratch. */
g4_status g4_cost_features(g4_tree tree, const float *aold_sorted, const uint8_t *bins_sorted,
                           const g4_params *params, float *features, int32_t *leaf_scratch,
                           void *stream);

/* Cost labels from the counts of the last walk: labels[i] = log(1 + PP_i + c_pn * PN_i).
 * counts: 2 x n uint32 as written by g4_gravity_tree. */
g4_status g4_cost_labels(const uint32_t *counts, int64_t n, float c_pn, float *labels, void *stream);

/* Inference: out[i] = MLP(features[i]) with BF16 weights and activations, FP32 sums. */
g4_status g4_mlp_forward(const float *params, const float *features, int64_t n, float *out,
                         void *stream);

/* Bytes of device workspace for g4_mlp_train_step on n samples. */
g4_status g4_mlp_train_workspace(int64_t n, size_t *bytes);

/* One Adam step (beta 0.9/0.999, eps 1e-8, bias-corrected with `step` >= 1) on the mean
 * squared error between MLP(features) and labels over all n samples; params, adam_m, adam_v:
 * g4_mlp_param_count() floats each (device, FP32 masters, updated in place).  lr = 0 only
 * computes the gradient.  loss_out (1 float) and grad_out (param count floats) are device
 * pointers and may be NULL.  The gradient is reduced in a fixed order (deterministic). */
g4_status g4_mlp_train_step(float *params, float *adam_m, float *adam_v, int32_t step,
                            const float *features, const float *labels, int64_t n, float lr,
                            float *loss_out, float *grad_out, void *workspace,
                            size_t workspace_bytes, void *stream);

/* Bytes of device workspace for g4_schedule_lpt with n sinks. */
g4_status g4_schedule_workspace(int64_t n, size_t *bytes);

/* Longest-processing-time schedule of the walk: group g holds sorted sinks [32g, 32g+32);
 * groups are taken in chunks of `chunk` consecutive groups (chunk = 1: single groups), a
 * chunk's predicted cost is the sum of expm1(pred) over its sinks, and group_order
 * (ceil(n/32) int32, device) lists the chunks by descending cost with the groups of a chunk
 * in PH order (chunks keep neighbouring groups together, which preserves cache reuse). */
g4_status g4_schedule_lpt(const float *pred_sorted, int64_t n, int32_t chunk, int32_t *group_order,
                          void *workspace, size_t workspace_bytes, void *stream);

/* Makes later g4_gravity_tree calls on this handle hand out groups in `group_order`
 * (device array of ngroups = ceil(n/32) entries, kept by pointer; NULL restores PH order).
 * Used only for whole-set walks of a single system whose group count matches. */
g4_status g4_tree_set_group_order(g4_tree tree, const int32_t *group_order, int64_t ngroups);

/* Bytes of device workspace for g4_schedule_items with n sinks. */
g4_status g4_schedule_items_workspace(int64_t n, size_t *bytes);

/* Partition of the walk by predicted cost (Sec. 6.1 balances the work with q_i, the
 * interactions of a particle's last force computation; here the prediction of the cost model
 * or the measured counts).  Group g (sorted sinks [32g, 32g+32)) has predicted cost
 * c_g = sum of expm1(max(pred, 0)) over its sinks.  A group with c_g > total / target (total =
 * sum of all c_g, fixed-order reduction) is split into K in {2, 4, 8} parts, K the smallest
 * power of two with c_g / K <= total / target: part k walks the tree for the same 32 sinks and
 * evaluates every K-th source of the group's source list (list positions k, k + K, ...), part 0
 * also the multipoles; the last part to finish adds the parts' sums in part order
 * (deterministic) and writes the outputs.  At most max_split groups are split (the first ones
 * in sink order); a large workload has c_g << total/target and is not split.  Items are ordered
 * by descending predicted part cost (stable).
 *   pred:    n floats (device): log(1 + cost) per sorted sink (cost model or measured labels).
 *   target:  desired number of equal-cost items (e.g. four per resident warp).
 *   items:   4 x 8 ceil(n/32) int32 (device): (first sink, count, part | parts << 8, split
 *            slot or -1); n_items: 1 int32 (device) = the number of valid items (the rest zero).
 * Every sink's interaction set is unchanged; sums round differently (other summation order). */
g4_status g4_schedule_items(const float *pred_sorted, int64_t n, int32_t target, int32_t max_split,
                            int32_t *items, int32_t *n_items, void *workspace,
                            size_t workspace_bytes, void *stream);

/* Makes later FP32 g4_gravity_tree calls on this handle take their work from `items` (device,
 * kept by pointer, as written by g4_schedule_items with the same max_split; n_items read on the
 * device) instead of fixed 32-sink groups.  capacity = number of items in the array.  Allocates
 * the partial-sum buffers of max_split split groups (6 KB each) when they grow, so call it
 * outside graph capture.  NULL restores the plain groups.  Used only for whole-set walks of a
 * single system (no active list, no forest) with n_sinks sinks; a malformed item sets the
 * list-capacity flag reported by g4_tree_status. */
g4_status g4_tree_set_work_items(g4_tree tree, const int32_t *items, const int32_t *n_items,
                                 int64_t capacity, int64_t n_sinks, int32_t max_split);

/* ---- helper: direct summation on the GPU --------------------------------------------------- */

/* O(n * n_sinks) direct sum with the same pair kernel (nearest image when periodic, pair
 * cutoff when TreePM and pp_cut).  sinks == NULL -> all particles.  acc 3 x n SoA, pot n. */
g4_status g4_direct(const uint32_t *pos, const float *mass, const uint8_t *cls, int64_t n,
                    const int32_t *sinks, int64_t n_sinks, const g4_params *params, float *acc,
                    float *pot, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* G4_H */
