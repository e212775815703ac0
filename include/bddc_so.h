/*
 * bddc_so.h -- C ABI of the GB300 (sm_103a) BDDC-SO library.
 *
 * BDDC-SO (Badia, Martin, Nguyen, "Balancing domain decomposition by
 * constraints associated with subobjects", arXiv 2001.07289) as the
 * preconditioner of PCG for Q1 finite-element diffusion
 *     -div(alpha grad u) = f on [0, nx h] x [0, ny h] x [0, nz h],
 *     u = 0 on the whole boundary
 * (Section 2, eq. weakform; Remark 1 for the per-element alpha; Section 5 for
 * the unit cube, f and the PCG stopping rule).
 *
 * Conventions shared by every entry point:
 *   - Node vectors are FP64 arrays of (nx+1)*(ny+1)*(nz+1) entries, node
 *     (i, j, k) at i + (nx+1)*(j + (ny+1)*k).  Entries on the Dirichlet
 *     boundary are ignored on input and written as 0 on output.
 *   - alpha is an FP64 array of nx*ny*nz entries, element (i, j, k) at
 *     i + nx*(j + ny*k), every entry finite and > 0.
 *   - Pointers named *_dev are device memory owned by the caller and must stay
 *     valid until the work queued on `stream` has finished; *_host pointers
 *     are ordinary host memory.  The library never frees caller memory.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  All device work is queued on it in order; entry points that
 *     return values to the host (pcg_solve, bddc_setup) synchronise it.
 *   - Every entry point returns 0 (BDDC_OK) or a negative BDDC_ERR_* code and
 *     never throws; bddc_last_error() gives a message for the last failure on
 *     a handle.  After BDDC_ERR_CUDA the handle should be destroyed.
 *   - One GPU: the device current when bddc_setup is called is used for the
 *     handle's whole life.  A handle is not thread-safe.
 */
#ifndef BDDC_SO_H
#define BDDC_SO_H

#ifdef __cplusplus
extern "C" {
#endif

enum {
    BDDC_OK = 0,
    BDDC_ERR_ARG = -1,        /* invalid sizes, cuts, L, options or alpha      */
    BDDC_ERR_NOT_SPD = -2,    /* non-positive pivot in a local or coarse factor */
    BDDC_ERR_NOCONV = -3,     /* PCG reached maxit before the tolerance         */
    BDDC_ERR_BREAKDOWN = -4,  /* PCG: p^T A p <= 0 or not finite                */
    BDDC_ERR_CUDA = -5,       /* a CUDA runtime call failed                     */
    BDDC_ERR_OOM = -6,        /* device allocation failed                       */
    BDDC_ERR_TIMEOUT = -7,    /* a bounded device wait gave up                  */
    BDDC_ERR_UNSUPPORTED = -8 /* valid request this build does not implement    */
};

/* Precision of the local factors and solves (the outer PCG, the weights and
 * the coarse problem are FP64 either way).  BDDC_MIXED keeps the local
 * factors in FP32, whose error grows with the local condition number: a
 * high-contrast inclusion that crosses a subdomain with few constraints on
 * it (thin channels of contrast 1e4 with Theta-hat = Theta, or with faces
 * only) can leave PCG without a usable preconditioner, while contrast 1e6 in
 * blocks aligned with many subobjects works; use BDDC_FP64 when in doubt. */
enum { BDDC_FP64 = 0, BDDC_MIXED = 1 };
enum { BDDC_W_CARD = 0, BDDC_W_RHO = 1 };    /* eq. (W) / Remark 1 weighting     */
/* Constraint selection (Table 1, Section 5): which objects of Theta-hat on
 * Gamma carry coarse DOFs.  VEF: vertices, edges and faces; VE: vertices and
 * edges; VF: vertices and faces; V: vertices only; F: faces only (the
 * BDDC-SO(f) of Section 5.2); EF: edges and faces.  Vertices, when selected,
 * are eliminated as primal DOFs; without them the local Neumann matrix of a
 * floating subdomain (no face on the Dirichlet boundary) is singular, so its
 * factor holds A + sum_k rho_k c_k^T c_k over the averages c_k lying in one
 * z-plane (an augmented Lagrangian: the constrained solves are unchanged and
 * the local coarse matrix loses rho_k on its diagonal).  Such a subdomain
 * without an average in one z-plane gives BDDC_ERR_UNSUPPORTED at setup.
 * The remark after Theorem 1 names
 * all edge or all face subobjects as sufficient for acceptable paths and all
 * vertex constraints as scalable but weaker, which the iteration counts show. */
enum { BDDC_SEL_VEF = 0, BDDC_SEL_VE = 1, BDDC_SEL_VF = 2, BDDC_SEL_V = 3, BDDC_SEL_F = 4, BDDC_SEL_EF = 5 };

typedef struct bddc_handle bddc_handle;

/* Structured mesh: nx*ny*nz cubes of side h (h <= 0 means h = 1/nx). */
typedef struct {
    int nx, ny, nz;
    double h;
} bddc_mesh;

/* Box partition Theta (Section 3): on axis d the subdomains are the slabs
 * between the ncut[d] interior cut planes cut[d][0] < ... (element indices in
 * (0, n_d)).  cut[d] is a host array; ncut[d] = 0 means one slab.
 *
 * Sub-partition Theta-hat: piece == NULL gives the boxes of the remark on
 * local subdivision in Section 3 (each subdomain side cut into pieces of at
 * most options.L_elems elements).  Otherwise piece is a host array of
 * nx*ny*nz sub-subdomain labels (x fastest, >= 0; elements with equal
 * labels form one sub-subdomain, which must lie in one subdomain, else
 * BDDC_ERR_ARG), e.g. material regions (Remark 1: a coefficient constant on
 * each sub-subdomain).  The (sub)objects are then the connected sets of
 * interface nodes with equal sets of surrounding sub-subdomains, typed by the
 * size of that set (2 face, 3 or 4 edge, more vertex); one-node vertices are
 * point values, every other object an average.  Read during the call only. */
typedef struct {
    int ncut[3];
    const int* cut[3];
    const int* piece;
} bddc_partition;

/* Options.  L_elems is the sub-object size L/h >= 1: every subdomain side of
 * w elements is split into ceil(w/L) pieces with boundaries floor(k w / s)
 * (Section 3: the sub-partition Theta-hat of characteristic size L). */
typedef struct {
    int precision;  /* BDDC_FP64 or BDDC_MIXED (FP32 local factors/solves, FP64 rest) */
    int weights;    /* BDDC_W_CARD or BDDC_W_RHO                                      */
    int L_elems;    /* >= 1                                                           */
    int selection;  /* BDDC_SEL_VEF, _VE, _VF, _V, _F or _EF                       */
    int use_graph;  /* 1: pcg_solve runs its whole loop as one CUDA graph (below)      */
    int maxit;      /* PCG iteration limit (<= 0: 2000)                               */
    int beta_rule;  /* BDDC_BETA_STANDARD (0) or BDDC_BETA_FLEXIBLE (below)          */
    int ml_block;   /* 0: exact coarse solve; g >= 1: multilevel BDDC-SO (below)     */
    int ml_sub;     /* multilevel: sub-block width s for level-2 subobjects (0: none) */
} bddc_options;

/* Multilevel BDDC-SO (Section 6: the multilevel version removes the coarse
 * problem's size limit).  With ml_block = g >= 1 the coarse problem is not
 * factored: each apply preconditions it by one application of BDDC on the
 * coarse level (Definition 1 once more), whose subdomains are blocks of
 * g x g x g subdomains (the last block of an axis takes the rest), whose
 * elements are the subdomains' local coarse matrices Phi_i^T A_i Phi_i, whose
 * interface holds the coarse DOFs shared by two or more blocks, grouped into
 * level-2 objects by the set of blocks sharing them (one constraint each: the
 * mean of the object's coarse values), with weights 1 / (blocks sharing the
 * DOF) (BDDC_W_CARD) or diagonal stiffness scaling, the coarse-level analogue
 * of Remark 1 (BDDC_W_RHO), and an exact level-2 coarse solve (by fronts of a
 * nested dissection of the block grid).  ml_sub = s >= 1 puts subobjects on
 * the coarse level, as Section 6 suggests: every block is cut into sub-blocks
 * of s x s x s subdomains and the level-2 objects group the interface coarse
 * DOFs by the set of sub-blocks sharing them (more level-2 coarse DOFs, fewer
 * PCG iterations).  All of it FP64.  B stays SPD;
 * the PCG iteration count grows (the condition number gains the coarse
 * level's factor) while the coarse set-up and solve shrink.  Its work
 * vectors are allocated at setup, so the allocation-free apply takes it too. */

/* PCG direction update p = z + beta p.  STANDARD (Section 5's PCG): beta =
 * r_{k+1}.z_{k+1} / r_k.z_k.  FLEXIBLE (Polak-Ribiere): beta =
 * r_{k+1}.(z_{k+1} - z_k) / r_k.z_k, one more dot product and node vector per
 * iteration; the same in exact arithmetic for a symmetric B (r_{k+1}.z_k = 0),
 * more robust when B varies between applications.  On the FP32-local path the
 * two take the same number of iterations on the workloads tested here. */
enum { BDDC_BETA_STANDARD = 0, BDDC_BETA_FLEXIBLE = 1 };

/* Per-solve statistics.  alphas/betas: optional host arrays of `capacity`
 * entries that receive the CG coefficients (for Lanczos estimates). */
typedef struct {
    int iterations;      /* operator applications after the initial residual */
    int converged;       /* 1 if ||r||_2 <= rtol ||b||_2                      */
    double r0_norm;      /* ||b||_2                                           */
    double r_norm;       /* final ||r||_2                                     */
    double* alphas;      /* in: host buffer or NULL; out: alpha_0..            */
    double* betas;       /* in: host buffer or NULL; out: beta_0..             */
    int capacity;        /* entries available in alphas/betas                 */
    double solve_ms;     /* device time of the solve (CUDA events)            */
} bddc_stats;

/* Sizes of a set-up preconditioner. */
typedef struct {
    int n_sub;            /* subdomains                                        */
    int n_coarse;         /* global coarse DOFs (objects carrying constraints) */
    int n_vertices;       /* of which point values                             */
    int max_local_coarse; /* largest n_c,i                                     */
    long long n_free;     /* non-Dirichlet nodes                               */
    long long bytes;      /* device memory held by the handle                  */
    long long factor_bytes;  /* local factors + Phi + coarse factor            */
    double setup_ms;      /* device time of bddc_setup (CUDA events)          */
    double phase_ms[6];   /* setup phases: 0 checks+weights, 1 local assembly,
                             2 local Dirichlet and Neumann factorisations (run
                             together), 3 coarse basis, 4 coarse assembly,
                             5 coarse Cholesky                                 */
    long long launches;   /* kernels launched for this handle since its setup
                             began (setup, applies, solves, gradients)        */
    double coarse_fma;    /* multiply-adds of the coarse factorisation         */
    double local_factor_fma;  /* multiply-adds of the local factorisations (inverse
                                 Schur complements of the plane blocks)           */
    long long apply_bytes;    /* bytes one bddc_apply must read from HBM: local
                                 factors (Dirichlet twice), Phi twice, coarse fronts */
    int apply_cluster;        /* CTAs per subdomain in the apply's local solves,
                                 chosen by timing (see bddc_setup)                 */
    double local_band_flops;  /* flops of banded Cholesky factorisations of the same
                                 local matrices: sum over subdomains of n_I b_I^2 +
                                 n_N b_N^2 (n free nodes, b = p_x p_y + p_x + 1 the
                                 lexicographic half-bandwidth, p free nodes per axis);
                                 the method-level count the roofline is quoted on   */
    int factor_kernel;        /* 1 if the tensor cores factored the subdomains whose
                                 planes fit them (FP32 path, tuned against the
                                 CUDA-core sweep), 0 if the CUDA cores did all      */
    int factor_tc_subdomains; /* subdomains factored on the tensor cores           */
    int pinned_subdomains;    /* floating subdomains without a point value, whose
                                 factors carry the augmented-Lagrangian terms      */
    int n_buckets;            /* non-empty size buckets of the apply's local solves */
    int bucket_subdomains[2]; /* per bucket: its subdomains (bucket 0: those whose
                                 work vectors need a whole SM, bucket 1: the rest)  */
    int bucket_ring[2];       /* per bucket: depth of the bulk-copy ring (6: one
                                 CTA per SM, 4: two), tuned                         */
    int bucket_ctas[2];       /* per bucket: CTAs per subdomain (1, 2 or 4), tuned   */
    int ml_blocks;            /* multilevel: blocks of the coarse level (0: exact coarse solve) */
    int ml_coarse2;           /* multilevel: level-2 coarse DOFs (level-2 objects)  */
} bddc_info_t;

/* Host-only analysis of a problem, no GPU needed: the counts that bddc_setup
 * would produce for the same arguments. */
typedef struct {
    int n_sub;            /* subdomains                                        */
    int n_coarse;         /* coarse DOFs: vertices + edges + faces of Theta-hat on Gamma */
    int n_vertices, n_edges, n_faces;  /* by object type (points on 3/2/1 axes) */
    int max_local_coarse; /* largest n_c,i                                     */
    int n_fronts;         /* fronts of the nested-dissection coarse Cholesky   */
    int n_levels;         /* depth of its front tree                           */
    int max_front;        /* largest front (pivots + update set)               */
    long long front_entries;  /* sum of squared front sizes (FP64 storage)    */
    double coarse_fma;    /* multiply-adds of the coarse factorisation         */
    int ml_blocks;        /* multilevel (options.ml_block > 0): blocks of the coarse level, else 0 */
    int ml_coarse2;       /* multilevel: level-2 coarse DOFs (level-2 objects)  */
    int ml_fronts2;       /* multilevel: fronts of the level-2 coarse Cholesky  */
} bddc_analysis_t;

/* Partition, sub-partition (Section 3 remark on local subdivision), object
 * classification and the coarse elimination plan, on the host.  Errors:
 * BDDC_ERR_ARG for invalid sizes, cuts or options. */
int bddc_analyze(const bddc_mesh* mesh, const bddc_partition* part,
                 const bddc_options* opt, bddc_analysis_t* out);

/* Acceptable-path check (remark after Theorem 1: the bound rests on the
 * auxiliary BDDC-A having, for every pair of neighbouring sub-subdomains, an
 * acceptable path; all edge or all face subobjects on Gamma guarantee one).
 * Host only; alpha_host (nx*ny*nz elements, x fastest, may be NULL for
 * alpha = 1) gives each sub-subdomain rho = the mean of alpha over it.
 * A pair is two sub-subdomains of different subdomains around one interface
 * node off the Dirichlet boundary.  It is direct when it shares a selected
 * edge or face object, or when every free node the two share is primal.
 * Otherwise it needs a path of sub-subdomains in which consecutive ones share
 * a face and either lie in one subdomain (continuity) or share a selected
 * face object or only primal free nodes; the path's quality is min(1, min of
 * rho over the path / min(rho_i, rho_j)) and the pair takes its best path's.
 * Sub-subdomains are those of the partition (boxes of size L or labels).
 * Errors: BDDC_ERR_ARG as bddc_analyze; BDDC_ERR_UNSUPPORTED above 2^22
 * sub-subdomains. */
typedef struct {
    long long n_pieces;        /* sub-subdomains                               */
    long long n_pairs;         /* neighbouring pairs across Gamma              */
    long long n_direct;        /* of which share a selected edge or face       */
    long long n_without_path;  /* of which have no acceptable path             */
    double min_ratio;          /* smallest best-path quality of the others (1 if none) */
    long long worst_pair[2];   /* a pair without a path, else one of min_ratio
                                  (-1 -1 when every pair is direct);
                                  sub-subdomain ids: box pieces a + na (b +
                                  nb c) of the per-axis piece indices, labels
                                  renumbered by first element               */
} bddc_paths_t;

int bddc_acceptable_paths(const bddc_mesh* mesh, const bddc_partition* part, const bddc_options* opt,
                          const double* alpha_host, bddc_paths_t* out);

/* Builds the BDDC-SO preconditioner (Section 3; Definition 1 with V1 = U_I,
 * Q1 = I, V2 = W-tilde, Q2 = (I - P)E): sub-partition and (sub)object
 * classification, weights of eq. (W) or Remark 1, local Dirichlet and
 * constrained Neumann factorisations, coarse basis Phi_i, coarse matrix and
 * its FP64 Cholesky factor.  Coarse objects are the vertices, edges and faces
 * of Theta-hat on Gamma; a vertex is a point value, an edge or face the mean
 * over its nodes.  alpha_dev is read during the call only.  On success *out
 * receives a new handle.  Errors: BDDC_ERR_ARG (bad sizes/cuts/L/options,
 * alpha <= 0 or not finite), BDDC_ERR_NOT_SPD, BDDC_ERR_OOM, BDDC_ERR_CUDA. *
 * Batching: the apply's per-subdomain kernels run in two size buckets (those
 * whose work vectors leave room for two CTAs per SM with a shallow bulk-copy
 * ring, and the rest), each one persistent launch per kernel, subdomains
 * longest first.  Autotuning: the first setup of a problem shape (precision,
 * subdomain count, largest planes, largest local coarse space, bucket sizes)
 * in the process times five preconditioner applies per candidate schedule of
 * each bucket (ring depth 6 or 4, one, two or four CTAs per subdomain) and
 * keeps the fastest (the default, ring depth 6 and one CTA, unless another is
 * at least 3 % faster) for every later handle of that shape; that first setup
 * takes up to about 72 applies longer. */
int bddc_setup(const bddc_mesh* mesh, const bddc_partition* part,
               const bddc_options* opt, const double* alpha_dev, void* stream,
               bddc_handle** out);

/* z = B r (Definition 1, Section 3): interior correction, weighted restriction
 * of the interface residual, coarse solve, constrained Neumann solves,
 * weighted injection E and discrete harmonic extension (I - P).  r_dev, z_dev:
 * node vectors (must not alias). */
int bddc_apply(bddc_handle* h, const double* r_dev, double* z_dev, void* stream);

/* y = A x, the matrix-free Dirichlet Q1 operator (Section 2 with Remark 1's
 * alpha).  x_dev, y_dev: node vectors (must not alias). */
int bddc_operator(bddc_handle* h, const double* x_dev, double* y_dev, void* stream);

/* PCG with preconditioner B from x0 = 0, stopped when ||r||_2 <= rtol ||b||_2
 * (Section 5: reduction of the residual 2-norm).  x_dev receives the iterate;
 * stats (may be NULL) the counts and coefficients.  Returns BDDC_OK,
 * BDDC_ERR_NOCONV (x holds the last iterate) or BDDC_ERR_BREAKDOWN.
 * The scalars and the stopping test stay on the device.  With
 * options.use_graph = 0 the host launches one iteration at a time and reads
 * the control flags after each; with use_graph = 1 the first solve on the
 * handle captures one iteration as the body of a graph while-loop (a
 * conditional node, ended by the device-side test, at most maxit times) on a
 * private stream, and every solve launches that graph once on `stream` with
 * no host round trip until the end.  Both modes launch the same kernels in
 * the same order and return bitwise identical results.  The graph lives in
 * the handle and is freed by bddc_destroy. */
int pcg_solve(bddc_handle* h, const double* b_dev, double* x_dev, double rtol,
              bddc_stats* stats, void* stream);

/* g_e = -h lambda_e^T K u_e per element: the derivative of J(u(alpha)) with
 * respect to alpha_e when A lambda = dJ/du (A is linear in alpha_e, Remark 1).
 * u_dev, lambda_dev: node vectors; g_dev: nx*ny*nz entries. */
int bddc_gradient(bddc_handle* h, const double* u_dev, const double* lambda_dev,
                  double* g_dev, void* stream);

/* The whole job from host memory: copies alpha and b to the device, runs
 * bddc_setup and pcg_solve, copies x back and frees everything it allocated.
 * For callers without device buffers and for end-to-end timing. */
int bddc_solve_host(const bddc_mesh* mesh, const bddc_partition* part,
                    const bddc_options* opt, const double* alpha_host,
                    const double* b_host, double* x_host, double rtol,
                    bddc_stats* stats);

/* Sizes and timings of a handle. */
int bddc_get_info(const bddc_handle* h, bddc_info_t* info);

/* Overrides the autotuned apply schedule of a handle: ctas_per_subdomain = 1,
 * 2 or 4 CTAs per subdomain in the local solves of bddc_apply (2, 4: a
 * thread-block cluster whose CTAs share each slot's rows), in every size
 * bucket.  All give the same preconditioner up to the summation order of the
 * partial sums.
 * Drops the handle's captured PCG graph (recaptured by the next pcg_solve).
 * The paper has no counterpart; BDDC_ERR_ARG for other values. */
int bddc_set_apply_schedule(bddc_handle* h, int ctas_per_subdomain);

/* The same for one size bucket (0 or 1, see bddc_info_t), with the depth of
 * its bulk-copy ring: 6 buffers (one CTA per SM) or 4 (two CTAs per SM, only
 * for a bucket whose work vectors fit).  The ring depth does not change the
 * arithmetic: results are bitwise the same.  BDDC_ERR_ARG for other values. */
int bddc_set_bucket_schedule(bddc_handle* h, int bucket, int ring_depth, int ctas_per_subdomain);

/* Copies the coarse basis of subdomain `sub` restricted to the subdomain's
 * box-surface nodes into phi_host (n_surface x n_c,i, row-major, FP64), the
 * global coarse numbers of its columns into gid_host and the box-surface node
 * ids into node_host; pass NULL buffers to query n_surface and n_c,i only.
 * Diagnostic access for tests. */
int bddc_get_coarse_basis(const bddc_handle* h, int sub, double* phi_host,
                          int* gid_host, long long* node_host,
                          int* n_surface, int* n_local_coarse);

/* Copies the assembled coarse matrix A_c (n_coarse^2, row-major, FP64, before
 * factorisation) to host memory; BDDC_ERR_UNSUPPORTED if it was not kept. */
int bddc_get_coarse_matrix(const bddc_handle* h, double* ac_host);

/* z = B r like bddc_apply, for callers that must not allocate device memory
 * while applying the preconditioner (code running under another framework's
 * memory pool, or solver loops that may not touch the CUDA allocator between
 * iterations).  The paper has no counterpart: this is a property of the
 * library.  It calls no cudaMalloc or cudaFree; all work vectors of the apply
 * live in one fixed 32 MiB device array that every GPU loading the library
 * holds until the process exits, and the handle's own buffers are not used.
 * Limits and behaviour:
 *   - problems whose apply work space exceeds 32 MiB (about 1.5 million mesh
 *     nodes in FP64) are rejected with BDDC_ERR_ARG and a message giving the
 *     size needed;
 *   - the first call on each device looks up the array's device address; make
 *     that first call before any stream capture;
 *   - every call, on every handle of the device, shares the one array, so
 *     calls whose GPU work overlaps (different streams, or concurrent host
 *     threads) race: order them on one stream;
 *   - the array keeps the last call's contents; each call clears what it needs
 *     zeroed.
 * Arguments as for bddc_apply. */
int bddc_apply_noalloc(bddc_handle* h, const double* r_dev, double* z_dev, void* stream);

/* Test hooks: host-side fault injection for the failure paths (the paper has
 * no counterpart).  Process-wide, not thread-safe; meant for tests only.
 *   BDDC_DEBUG_NEGATE_NEUMANN_PIVOT / _DIRICHLET_PIVOT, value = subdomain id
 *     (x fastest over the box grid; -1 = off): every later bddc_setup negates
 *     the first diagonal entry of that subdomain's assembled local Neumann
 *     (Dirichlet) matrix before factorising it, so the setup returns
 *     BDDC_ERR_NOT_SPD and bddc_last_error(NULL) names the subdomain.  A
 *     subdomain without interior nodes has no Dirichlet matrix: no effect.
 *   BDDC_DEBUG_WAIT_TRIES, value = tries (< 0: the default): every bounded
 *     device wait (bulk copies, tensor-core MMAs) reports a timeout after this
 *     many unsuccessful tries, then still waits, bounded, for the work it
 *     covers, so the results stay valid and nothing hangs; the next call that
 *     reads the device status (pcg_solve, bddc_setup) returns
 *     BDDC_ERR_TIMEOUT and clears it.  0 makes every wait report.
 *   BDDC_DEBUG_CLEAR: every hook off.
 * Returns BDDC_ERR_ARG for an unknown hook or value. */
enum { BDDC_DEBUG_CLEAR = 0, BDDC_DEBUG_NEGATE_NEUMANN_PIVOT = 1, BDDC_DEBUG_NEGATE_DIRICHLET_PIVOT = 2,
       BDDC_DEBUG_WAIT_TRIES = 3 };
int bddc_debug_inject(int what, long long value);

/* Frees every device and host resource of the handle (NULL is a no-op). */
int bddc_destroy(bddc_handle* h);

/* Message for the last error on the handle (or the last failed bddc_setup
 * when h is NULL).  Owned by the library. */
const char* bddc_last_error(const bddc_handle* h);

#ifdef __cplusplus
}
#endif
#endif /* BDDC_SO_H */
