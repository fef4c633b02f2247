/*
 * lrh.h — C ABI of the B300 message-passing dual solver for local relaxation
 * hierarchies of quantum ground-state energies.
 *
 * The library runs, on one GPU, the data-parallel iteration of the paper's
 * dual solvers over every region e of a cluster family C:
 *
 *   theta_e = h_e - sum_{f in D(e)} 1_{e\f} (x) nu_{e->f} + sum_{g in A(e)} nu_{g->e}
 *                                                        (Sec. 4.2, local augmented Hamiltonian)
 *   theta_e = V diag(lambda) V^dagger                    (Hermitian eigendecomposition, FP32)
 *   subgradient (Alg. 1):  mu_e = ground projector / its trace,  value lambda_min(theta_e)
 *   smoothed   (Alg. 2):  rho_e = V softmax(-beta lambda) V^dagger,
 *                         value F_beta = lambda_min - log(sum e^{-beta(lambda-lambda_min)}) / beta
 *                                                        (Sec. 4.1.2, soft local minimum eigenvalue)
 *   g_{e->f} = rho_f - Tr_{e\f} rho_e                    (Sec. 4.1.1 / 4.1.2 / 4.2 gradient components)
 *   Alg. 1 update:  nu += alpha_t g,  best-so-far q and nu tracked
 *   Alg. 2 update:  zeta += g / (theta_k L_hat),  nu = (1-theta_k) nu + theta_k zeta,
 *                   theta_{k+1} = (sqrt(theta_k^4 + 4 theta_k^2) - theta_k^2) / 2,
 *                   messages evaluated at eta = (1-theta_k) nu + theta_k zeta
 *   bound Q(nu) = sum_e lambda_min(theta_e(nu))           (Eq. dual_function_non-smooth; Q_C, Sec. 4.2)
 *                 summed in FP64; the certified bound rebuilds theta_e in FP64 from the stored
 *                 FP32 messages and takes lambda_min in FP64 (weak duality makes it a valid
 *                 lower bound on E_0 for any Hermitian nu).
 *
 * Conventions
 * -----------
 * - Every site is a qubit (local dimension d = 2).  A region with k sites has D = 2^k.
 * - Kronecker order inside a region (and inside a term): the region's sites sorted ascending,
 *   first site = most significant bit of the basis index.
 * - Pairs e->f are the covering relation of the region family under inclusion (f a proper
 *   subset of e with no region strictly between them; Sec. 4.2 remark that only consecutive
 *   levels need constraints).  Pair order: ascending parent index, then ascending child index.
 * - Message layout (all message-like arrays: nu, zeta, nu_best, gradient): per instance, the
 *   pairs in pair order, each a D_f x D_f complex matrix row-major, complex64 = (float re, float im).
 *   Instances are contiguous blocks of lrh_info.msg_elems complex entries.
 * - Term placement: each Hamiltonian term goes to the smallest region containing its sites
 *   (lowest region index on ties).
 *
 * Ownership and errors
 * --------------------
 * - Every pointer in lrh_problem_desc is a HOST pointer; the library copies what it needs
 *   during lrh_create and keeps no reference.
 * - The library owns all device memory of a problem; lrh_destroy frees it.
 * - Buffers passed to lrh_get_messages / lrh_set_messages belong to the caller; a device buffer
 *   must be on the problem's device.
 * - All calls return LRH_OK (0) or a negative LRH_E* code; no C++ exception crosses the ABI.
 *   lrh_last_error() returns a thread-local message describing the last failure.
 * - Work is enqueued on the stream given at creation (NULL = the legacy default stream);
 *   lrh_step returns without waiting.  Calls that return numbers to the host synchronise
 *   that stream.  A problem must not be used from two host threads at once.
 */
#ifndef LRH_H
#define LRH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- return codes */
#define LRH_OK            0
#define LRH_EINVAL       (-1)  /* bad argument, size or option */
#define LRH_ENOTHERM     (-2)  /* a term matrix is not Hermitian */
#define LRH_EPOSET       (-3)  /* duplicate region, or a term fits in no region */
#define LRH_ENOMEM       (-4)  /* host or device allocation failed */
#define LRH_ECUDA        (-5)  /* a CUDA runtime call failed */
#define LRH_ETIMEOUT     (-6)  /* a bounded device wait gave up (grid barrier of the persistent launch) */
#define LRH_ENUMERIC     (-7)  /* a non-finite eigenvalue, value or message was produced */
#define LRH_EUNSUPPORTED (-8)  /* region size beyond the kernels built into this library */
#define LRH_ENOCONV      (-9)  /* an FP64 certification eigensolve stopped at its sweep cap before
                                  converging; the bound returned with it is still a valid lower
                                  bound (Weyl-corrected), only looser */
#define LRH_EDEADLINE   (-10)  /* lrh_solve stopped at lrh_options.deadline_s (results are those of
                                  the last completed certification) */

/* ---------------------------------------------------------------- enums */
#define LRH_SUBGRADIENT   0    /* Alg. 1: ground projectors, nu += alpha_t g            */
#define LRH_NESTEROV      1    /* Alg. 2: Gibbs states at eta, accelerated update of Q_beta */

#define LRH_STEP_CONST    0    /* alpha_t = alpha                        (Thm 4 choice)  */
#define LRH_STEP_INV_SQRT 1    /* alpha_t = alpha / sqrt(t + 1)                           */

#define LRH_LOOP_EAGER      0  /* lrh_options.loop: one launch per kernel per iteration        */
#define LRH_LOOP_GRAPH      1  /* replay of a captured CUDA graph of iterations               */
#define LRH_LOOP_PERSISTENT 2  /* one cooperative launch for all iterations of an lrh_step    */
#define LRH_LOOP_AUTO       3  /* chosen by lrh_autotune (graph or persistent)                */

#define LRH_SHAPE_BLOCKS  4096  /* lrh_set_launch_shape, classes of 3-4 sites: LRH_SHAPE_BLOCKS + 64 / 128 / 256
                                   selects the Hermitian 2x2-block layout (theta's upper triangle in
                                   shared memory, each stored entry rotated once per round) with that
                                   many threads per CTA; D lanes per region as in the lane-row layout */
#define LRH_SHAPE_WARP16  8192  /* lrh_set_launch_shape, 4-site classes: LRH_SHAPE_WARP16 + 64 / 128 / 256
                                   selects the 2x2-block layout with one warp per 16 x 16 region (each
                                   lane one off-diagonal block and half a row of V) */
#define LRH_SHAPE_CTA_FP32   1  /* lrh_set_launch_shape, classes of 6-8 sites: rho = W W^dagger on the FP32 cores */
#define LRH_SHAPE_CTA_TENSOR 2  /* ... on the tensor cores (tcgen05, three TF32 products per term, FP32
                                   accumulate); 7-site (128 x 128) regions only */

#define LRH_MSG_NU        0    /* current multipliers nu                                  */
#define LRH_MSG_ZETA      1    /* Nesterov auxiliary sequence zeta                        */
#define LRH_MSG_NU_BEST   2    /* subgradient: nu at the best q seen so far               */
#define LRH_MSG_GRAD      3    /* gradient g of the last lrh_evaluate (read only)         */

#define LRH_BOUND_CERTIFIED 0  /* FP64 rebuild + FP64 lambda_min at nu (Alg. 2) or nu_best (Alg. 1) */
#define LRH_BOUND_LAST      1  /* FP64 sum of the per-region FP32 values of the last region pass:
                                  Q_beta(eta) for Alg. 2, Q(nu) for Alg. 1                   */
#define LRH_BOUND_BEST      2  /* Alg. 1 q_best = max over past iterations of Q(nu^(t))      */

/* The certified value of a region is min_i a_ii - ||offdiag(A)||_F of the matrix A the FP64
 * Jacobi iteration ends with (Weyl's inequality: a lower bound on lambda_min(theta) whether or
 * not the iteration converged; at convergence the correction is below 1e-14 ||theta||_F).  If a
 * region stopped at the sweep cap with ||offdiag||_F^2 > 1e-28 ||theta||_F^2, lrh_bound returns
 * LRH_ENOCONV and still fills `out`. */

/* ---------------------------------------------------------------- problem description */
typedef struct {
    int32_t n_sites;              /* sites 0 .. n_sites-1, all qubits                          */
    int32_t n_regions;            /* regions of the cluster family                             */
    const int64_t* region_ptr;    /* [n_regions + 1] CSR offsets into region_sites             */
    const int32_t* region_sites;  /* sorted, unique site ids of each region (1..8 sites)       */
    int32_t n_terms;              /* Hamiltonian terms                                          */
    const int64_t* term_ptr;      /* [n_terms + 1] CSR offsets into term_sites                 */
    const int32_t* term_sites;    /* sorted, unique sites of each term                          */
    const int64_t* term_mat_off;  /* [n_terms] offset (complex entries) of each term's matrix  */
    int64_t term_mat_total;       /* complex entries of all term matrices of ONE instance       */
    const double* term_mats;      /* [n_instances][term_mat_total][2] (re, im), row-major
                                     2^k x 2^k per term; instance i holds its own matrices     */
    int32_t n_instances;          /* >= 1 Hamiltonians sharing one region family (batch)       */
    /* Optional explicit pairs e -> f (n_pairs > 0): consistency constraints between region
     * pair_parent[q] and region pair_child[q], whose sites must be a proper subset of the
     * parent's; duplicates are rejected (LRH_EPOSET).  Any set of such pairs gives a valid
     * relaxation (Sec. 4.2 notes that the covering pairs suffice); they are stored in pair order
     * whatever order they are given in.  n_pairs = 0: the covering relation of inclusion.     */
    int64_t n_pairs;
    const int32_t* pair_parent;
    const int32_t* pair_child;
    /* Optional explicit term placement: term t is embedded into region term_region[t], which
     * must contain its sites (LRH_EPOSET otherwise).  NULL: the placement rule above.        */
    const int32_t* term_region;
    /* Optional ghost flags [n_regions] (nonzero = ghost) of one shard of a sharded lattice (see
     * lrh_halo_set): a ghost region's pass runs on another shard; this problem neither
     * computes it nor counts it in its bounds.  NULL: no ghosts.  Not every region may be a
     * ghost.                                                                                 */
    const uint8_t* region_ghost;
} lrh_problem_desc;

typedef struct {
    int32_t variant;      /* LRH_SUBGRADIENT or LRH_NESTEROV                                  */
    int32_t step_rule;    /* LRH_STEP_CONST or LRH_STEP_INV_SQRT (subgradient only)           */
    double  alpha;        /* subgradient step scale (> 0)                                     */
    double  beta;         /* smoothing inverse temperature (> 0, Nesterov)                    */
    double  lhat;         /* Lipschitz estimate L_hat; <= 0 selects beta * Lambda_G / 2       */
    double  degen_tol;    /* ground space = eigenvalues within degen_tol * max(1,||theta||_F)
                             of lambda_min (subgradient); <= 0 selects 1e-5                   */
    int32_t max_sweeps;   /* Jacobi sweep cap of the FP32 eigensolver; <= 0 selects 15 (regions
                             of 8 sites: at most 16, the sweeps their rotation log holds)   */
    int32_t loop;         /* iteration driver of lrh_step: LRH_LOOP_EAGER (kernel launches),
                             LRH_LOOP_GRAPH (a captured CUDA graph of iterations),
                             LRH_LOOP_PERSISTENT (one cooperative launch running all the
                             iterations, grid-wide barriers between passes; problems whose
                             classes all have <= 4 sites, else GRAPH), LRH_LOOP_AUTO (the
                             choice of lrh_autotune; GRAPH before it).  All drivers give
                             bit-identical messages for the same launch shapes; the
                             persistent one runs every class in the lane layout.             */
    int32_t cert_sweeps;  /* sweep cap of the FP64 certification eigensolver; <= 0 selects 40  */
    /* Schedule run by lrh_solve (all host values, copied by lrh_create / lrh_set_options):   */
    int32_t n_beta;              /* Alg. 2: beta-continuation stages (0: one stage at `beta`)  */
    const double* beta_sched;    /* [n_beta] stage inverse temperatures (> 0); each stage sets
                                    L_hat = lhat if lhat > 0 else beta_s Lambda_G / 2 and restarts
                                    (theta = 1, zeta = nu)                                     */
    int32_t iters_per_stage;     /* Alg. 2: iterations of every stage; Alg. 1: of the run      */
    int32_t certify_every;       /* lrh_solve records the certified bound every this many
                                    iterations (<= 0: at the end of the run only)              */
    double deadline_s;           /* lrh_solve stops at the first record after this many
                                    seconds of wall time (<= 0: no deadline)                  */
    const char* tune_cache;      /* cache file lrh_autotune uses when called with NULL (copied) */
    /* Target-driven solve (lrh_solve with certify_every > 0): */
    const double* target;        /* [n_instances] or NULL (copied): lrh_solve stops at the first
                                    checkpoint whose certified bound is >= target[i] on every
                                    instance i with a finite target                            */
    double screen_tol;           /* > 0 (with target): before certifying a checkpoint, estimate
                                    Q(nu) = sum_e lambda_min(theta_e) in FP32 (one region pass)
                                    and certify (FP64) only if the estimate is >= target[i] -
                                    screen_tol on every targeted instance; the run's last
                                    checkpoint is always certified.  0: certify every checkpoint */
    int32_t cold_start;          /* 0 (default): the FP32 eigensolve of a region of 3, 4, 6 or 7 sites
                                    starts from the eigenvectors its previous pass stored (one
                                    D x D basis per region and instance on the device, the
                                    identity at creation): theta_e is first rotated into that
                                    basis, after one Newton-Schulz step makes it unitary to
                                    rounding, and Jacobi sweeps only what theta_e moved since.
                                    Nonzero: every eigensolve starts from the identity and the
                                    stored bases are neither read nor written; nonzero at
                                    lrh_create allocates no bases at all (lrh_info.warm_bytes
                                    = 0), and the problem then stays cold whatever later
                                    options say.  Either way the eigensolve stops at the same
                                    threshold.                                                */
} lrh_options;

typedef struct lrh_problem lrh_problem;

typedef struct {
    int32_t n_instances;
    int32_t n_regions;            /* per instance                                              */
    int32_t n_pairs;              /* per instance                                              */
    int32_t max_region_sites;
    int64_t msg_elems;            /* complex entries of one instance's message array           */
    double  lambda_G;             /* Lambda_G of the L_hat rule (Delta_G + d at level 1,
                                     max_{e->f} m_f + m_e D_e/D_f otherwise; Thms 5 and 7)     */
    double  gamma_G;              /* Gamma_G = sum_e log D_e (smoothing-error lemma)           */
    int64_t iteration;            /* iterations run since creation                             */
    int32_t n_classes;            /* region size classes present                               */
    int32_t class_sites[8];       /* k of each class                                           */
    int32_t class_regions[8];     /* regions per instance of each class                        */
    uint64_t sweeps[8];           /* cumulative FP32 Jacobi sweeps x regions, per class        */
    int32_t class_block[8];       /* threads per CTA of each class's region pass (autotuned);
                                     negative: one thread per region (4 x 4 regions); classes of
                                     6-8 sites: LRH_SHAPE_CTA_FP32 / LRH_SHAPE_CTA_TENSOR        */
    int32_t concurrent_classes;   /* region classes of one pass: 0 one after another, 1 on forked
                                     streams, 2 in one launch (classes of <= 4 sites; autotuned) */
    int32_t loop;                 /* driver lrh_step uses now (LRH_LOOP_EAGER/GRAPH/PERSISTENT)  */
    int32_t persistent_grid;      /* CTAs of the persistent launch (0: not available)             */
    int64_t persistent_tiles;     /* region tiles per pass in the persistent launch               */
    uint64_t sweep_capped[8];     /* cumulative FP32 eigensolves per class that stopped at
                                     lrh_options.max_sweeps before reaching the threshold
                                     ||offdiag||_F^2 <= 1e-12 ||theta||_F^2                      */
    int32_t n_sites;
    int32_t kappa_G;              /* max over sites i of |{e->f : i in f}| (Thm 6; Delta_G at level 1) */
    int64_t warm_bytes;           /* device bytes of the stored eigenbases (lrh_options.cold_start) */
} lrh_info;

/* Parameter rules of the convergence theorems for a target error density eps (per site):
 *   Alg. 2 (Thm 5, Thm 7): beta = 2 Gamma_G / (n eps), L_hat = beta Lambda_G / 2,
 *                          T >= ceil(2 R sqrt(Gamma_G Lambda_G) / (n eps)) - 1;
 *   Alg. 1 (Thm 4, Thm 6): alpha = c eps with c = c_frac / kappa_G (0 < c_frac < 1),
 *                          T >= ceil(R^2 / (2 c (1 - c kappa_G) n eps^2)).
 * R is the distance from nu^(0) to the optimal multipliers (caller's estimate; <= 0: the
 * iteration counts are returned as -1).  Lambda_G is Delta_G + d for pure level-1 posets and
 * max_{e->f} (m_f + m_e D_e / D_f) otherwise (the two lemmas on L_hat). */
typedef struct {
    double beta, lhat, alpha, c;
    double lambda_G, gamma_G;
    int32_t kappa_G;
    int32_t n_sites;
    int64_t T_nesterov, T_subgradient;
} lrh_params;

/* One record of lrh_solve: the certified bound after `iteration` iterations of the run (with
 * screening, only the checkpoints that were certified are recorded). */
typedef struct {
    int64_t iteration;   /* iterations since the start of this lrh_solve call               */
    double seconds;      /* host wall time since the start of the call, after the bound was read */
    double beta;         /* stage inverse temperature (Alg. 2; 0 for Alg. 1)                */
} lrh_record;

/* ---------------------------------------------------------------- entry points */

/* Build the region poset, place and embed the terms, allocate device state and zero the
 * messages (Alg. 1 / Alg. 2 initialisation nu = zeta = 0, theta_0 = 1).  `stream` is a
 * cudaStream_t (or NULL) on the current device.  On failure *out is NULL. */
int lrh_create(const lrh_problem_desc* desc, const lrh_options* opts, void* stream,
               lrh_problem** out);

/* Free all host and device memory of the problem (NULL is accepted). */
void lrh_destroy(lrh_problem* p);

/* Sizes, constants and counters (host only, no synchronisation). */
int lrh_get_info(const lrh_problem* p, lrh_info* info);

/* Pair table in pair order: parent, child region ids and the complex offset of each
 * message inside one instance's message array.  Each output may be NULL; arrays hold
 * lrh_info.n_pairs entries. */
int lrh_get_pairs(const lrh_problem* p, int32_t* parent, int32_t* child, int64_t* msg_off);

/* Replace the options (beta / L_hat / alpha / rule / tolerances).  Stream-ordered. */
int lrh_set_options(lrh_problem* p, const lrh_options* opts);

/* Start a new smoothing stage: theta = 1 and zeta = nu (beta-continuation restart), and
 * reset the step counter t used by LRH_STEP_INV_SQRT.  For LRH_SUBGRADIENT it also starts a
 * new best-so-far record (q_best = -inf).  Stream-ordered (synchronises for LRH_SUBGRADIENT). */
int lrh_restart(lrh_problem* p);

/* Run n_iters iterations of the selected algorithm (asynchronous). */
int lrh_step(lrh_problem* p, int32_t n_iters);

/* One region pass at the current point without updating any message: stores the per-region
 * values and the gradient g (readable with LRH_MSG_GRAD / lrh_get_region_values).
 * Alg. 2 evaluates at eta = (1-theta) nu + theta zeta, Alg. 1 at nu. Asynchronous. */
int lrh_evaluate(lrh_problem* p);

/* Enqueue only the region pass of one size class (regions with k_sites sites, all instances)
 * at the current point, without any message update: assembly, FP32 eigendecomposition,
 * state, partial traces and per-region values of that class.  Used to time the dominant
 * kernel of an iteration on the problem's stream.  Returns LRH_EINVAL if no region has
 * k_sites sites. Asynchronous. */
int lrh_launch_region_pass(lrh_problem* p, int32_t k_sites);

/* Per-instance bound of the requested kind into out[n_instances] (host). Synchronises. */
int lrh_bound(lrh_problem* p, int32_t kind, double* out);

/* Per-region values [n_instances][n_regions] (host): kind LRH_BOUND_LAST gives the FP32
 * pass values (F_beta or lambda_min), LRH_BOUND_CERTIFIED the FP64 lambda_min of the last
 * certification. Synchronises. */
int lrh_get_region_values(lrh_problem* p, int32_t kind, double* out);

/* Copy a message-like array out of / into the library.  `bytes` must equal
 * n_instances * msg_elems * 8.  dst/src is a device pointer when *_is_device is nonzero.
 * lrh_set_messages rejects LRH_MSG_GRAD and symmetrises nothing: the caller provides
 * Hermitian blocks. Stream-ordered (get synchronises when dst is on the host). */
int lrh_get_messages(lrh_problem* p, int32_t which, void* dst, int64_t bytes, int32_t dst_is_device);
int lrh_set_messages(lrh_problem* p, int32_t which, const void* src, int64_t bytes, int32_t src_is_device);

/* Replace the term matrices (same sites, offsets and instance count as at creation; host
 * pointer, layout of lrh_problem_desc.term_mats).  Used to differentiate with respect to
 * couplings.  Synchronises. */
int lrh_set_terms(lrh_problem* p, const double* term_mats);

/* Reverse-mode derivative (adjoint) of the smoothed evaluation done by lrh_evaluate, at the
 * same point eta = (1-theta) nu + theta zeta (Nesterov problems, regions of <= 5 sites).
 * The evaluation maps term matrices T and multipliers to Q_beta (per instance) and the
 * gradient g (message layout) (Sec. 4.1.2, 4.2).  Given cotangents q_bar (host double
 * [n_instances]) and g_bar (complex64 message layout, device if g_bar_is_device, NULL = 0)
 * it writes nu_bar (complex64, message layout) and term_bar (complex64, layout of the term
 * matrices, [n_instances][term_mat_total]) under the inner product Re Tr(A^dagger B):
 *   rho_bar_e = sum_parents g_bar - sum_children 1 (x) g_bar,
 *   theta_bar = V[(V^dagger rho_bar V) o K + (beta <rho_bar, rho> + q_bar) diag(p)] V^dagger,
 *   K_kl = (p_k - p_l)/(lambda_k - lambda_l), K_kk = -beta p_k  (eigenbasis recomputed),
 *   nu_bar_{e->f} = theta_bar_f - Tr_{e\f} theta_bar_e,  term_bar_t = Tr_{R\t} theta_bar_R.
 * The derivative with respect to nu_{e->f} of eta-evaluated quantities is returned for eta
 * itself.  Outputs are device pointers when out_is_device (each may be NULL).
 * The first call allocates the adjoint buffers.  Synchronises. */
int lrh_vjp(lrh_problem* p, const double* q_bar, const void* g_bar, int32_t g_bar_is_device, void* nu_bar,
            void* term_bar, int32_t out_is_device);

/* Autotuner.  Times, on this problem's own data and stream, the launch shapes of every region
 * class with at most 5 sites (64, 128 or 256 threads per CTA, i.e. 64/D .. 256/D regions per
 * CTA), whether the classes of one pass run one after another, on forked streams or in one
 * launch, and, when
 * the problem allows a persistent launch, the graph against the persistent iteration driver
 * (used when lrh_options.loop is LRH_LOOP_AUTO); then keeps the fastest.  Choices are read
 * from / appended to `cache_path` (JSON lines keyed by class size, region count and SM count;
 * NULL = no cache); flags bit 0 forces re-measuring.  Classes of 3 and 4 sites with stored
 * eigenbases are tuned among the 2x2-block shapes only (the layout that warm-starts).  Runs region passes at the current point
 * (their outputs are recomputed by the next iteration) and iterations on a saved copy of the
 * multipliers, which it restores; the stored eigenbases (lrh_options.cold_start) are copied to
 * a temporary device buffer of lrh_info.warm_bytes and put back (LRH_ENOMEM if that buffer
 * cannot be had), so tuning does not change later results; must not be called during stream
 * capture; synchronises. */
int lrh_autotune(lrh_problem* p, const char* cache_path, int32_t flags);

/* Set the launch shape of one region class by hand (what lrh_autotune chooses): 64, 128 or
 * 256 threads per CTA with 2^k_sites lanes per region, or for 4 x 4 regions -64, -128, -256 for
 * one thread per region.  The lane layouts give bit-identical results; the one-thread layout
 * rotates in another order and agrees to rounding.  For classes of 6 to 8 sites (one CTA per
 * region) the shape selects the back-transform: LRH_SHAPE_CTA_FP32, or for 7 sites also
 * LRH_SHAPE_CTA_TENSOR (results agree to FP32 rounding). */
int lrh_set_launch_shape(lrh_problem* p, int32_t k_sites, int32_t block);

/* How the region classes of one pass are launched (what lrh_autotune chooses): 0 one class
 * after another on the problem's stream, 1 on forked streams (the default), 2 all classes in
 * one launch (problems whose classes all have <= 4 sites; LRH_EUNSUPPORTED otherwise).  All
 * three give bit-identical results for lane launch shapes. */
int lrh_set_class_mode(lrh_problem* p, int32_t mode);

/* Self-test of the bounded grid-barrier wait of the persistent driver: one persistent launch
 * whose first barrier is never released (it waits for one CTA more than the grid), so every CTA gives
 * up after the wait limit (one second) and raises the timeout status.  Returns LRH_ETIMEOUT
 * when the wait ended as designed (the status is then cleared and the problem stays usable;
 * the pass before the barrier only rewrites states and values that the next iteration
 * recomputes), LRH_EUNSUPPORTED when the problem has no persistent launch.  Synchronises. */
int lrh_selftest_barrier_timeout(lrh_problem* p);

/* Checkpoint / resume.  The state is the iteration scalars (theta_k, step counter, beta,
 * L_hat, alpha, iteration parity), nu, zeta, nu_best, q_best and the stored eigenbases of the
 * regions of 3, 4, 6 and 7 sites (lrh_options.cold_start; lrh_info.warm_bytes), packed into one host buffer
 * of lrh_state_bytes() bytes; lrh_set_state accepts only a buffer from a problem with the same
 * instance count, message layout and variant.  Resuming from a saved state and iterating gives
 * bit-identical messages to an uninterrupted run.  Both synchronise. */
int64_t lrh_state_bytes(const lrh_problem* p);
int lrh_get_state(lrh_problem* p, void* buf, int64_t bytes);
int lrh_set_state(lrh_problem* p, const void* buf, int64_t bytes);

/* Wait for the problem's stream and report any device-side numeric error (LRH_ENUMERIC). */
int lrh_synchronize(lrh_problem* p);

/* Allocation-free evaluation of a pairwise (level-1: edges + sites) smoothed dual.
 * The paper has no counterpart of this entry point; it exists for callers that cannot call
 * cudaMalloc (code inside another runtime's allocator or memory pool, processes whose device
 * memory is reserved up front) and therefore cannot use lrh_create.  It computes what
 * lrh_evaluate computes for a Nesterov problem whose regions are the given edges and all
 * sites (with eta = nu): Q_beta = sum of F_beta over edges and sites, and the gradient
 * g_{e->v} = rho_v - Tr_{e\v} rho_e, using only caller-owned buffers plus a fixed scratch
 * array compiled into the library (about 5 MB of device memory on every GPU that loads the
 * library, held until the process exits).  Limits: n_sites <= 65536, n_edges <= 131072;
 * larger sizes return LRH_EINVAL.
 *   edges    device int32 [n_edges][2]: two distinct sites 0 <= site < n_sites per edge; the
 *            first one is the most significant factor of the edge's 4 x 4 index.  An endpoint
 *            out of range or repeated is not used: the edge's gradient blocks and *value_out
 *            are set to NaN (the call still returns LRH_OK; the check runs on the device)
 *   h_edge   device complex64 [n_edges][4][4] edge terms in that order, or NULL (zero)
 *   h_site   device complex64 [n_sites][2][2] site terms, or NULL (zero)
 *   nu       device complex64 [n_edges][2][2][2]: nu_{e->first site}, then nu_{e->second site}
 *   beta     smoothing inverse temperature (> 0)
 *   value_out device double [1] receives Q_beta; grad_out device complex64 [n_edges][2][2][2]
 * Every matrix must be Hermitian (only upper triangles of 2 x 2 blocks are read for sites).
 * Each site sums its incoming messages in ascending edge order, so repeated calls with the same
 * inputs give bit-identical outputs.  Asynchronous on `stream` (a cudaStream_t or NULL).  Calls
 * share the scratch array: calls that may overlap on the GPU race and must be ordered by the
 * caller.  The first call on a device looks up the scratch address for that device; make it
 * before any stream capture.  Calls no allocating routine. */
int lrh_level1_eval_noalloc(int32_t n_sites, int32_t n_edges, const int32_t* edges, const void* h_edge,
                            const void* h_site, const void* nu, double beta, double* value_out,
                            void* grad_out, void* stream);

/* Theorem parameter rules (see lrh_params) for target error density eps > 0; host only. */
int lrh_theorem_parameters(const lrh_problem* p, double eps, double R, double c_frac, lrh_params* out);

/* Zero nu, zeta, nu_best (Alg. 1 / Alg. 2 initialisation), set theta = 1, t = 0,
 * q_best = -inf and every stored eigenbasis to the identity: the state at creation.
 * Stream-ordered. */
int lrh_reset(lrh_problem* p);

/* Run the schedule of lrh_options from the current multipliers: Alg. 2 runs one stage per
 * beta_sched entry (or one stage at `beta`), each stage setting beta and L_hat and restarting
 * (theta = 1, zeta = nu; reading of the paper: Alg. 2 with one fixed beta, continued over
 * stages), then iters_per_stage iterations; Alg. 1 restarts and runs iters_per_stage
 * iterations.  Every certify_every iterations (and at the end) the certified bound
 * (LRH_BOUND_CERTIFIED) is computed; up to max_records records are written to rec[] with the
 * per-instance bounds in rec_bounds[max_records][n_instances] (both host, may be NULL with
 * max_records = 0), their count to *n_records (may be NULL).  bound_out[n_instances] (host)
 * receives the last certified bound.  With deadline_s > 0 the run stops at the first record
 * taken after the deadline and returns LRH_EDEADLINE.  Synchronises at every record. */
int lrh_solve(lrh_problem* p, int32_t max_records, lrh_record* rec, double* rec_bounds, int32_t* n_records,
              double* bound_out);

/* Static message for an error code, and the thread-local detail of the last failure. */
const char* lrh_strerror(int code);
const char* lrh_last_error(void);

/* ---------------------------------------------------------------- sharding with halo exchange
 * One lattice split into shards, one problem (and GPU) per shard; Alg. 2 only.  The paper's
 * region and message loops are independent within an iteration (Alg. 1 and Alg. 2 mark them
 * parallel), so a shard needs from the others, per iteration, only the two inputs of the
 * gradient g_{e->f} = rho_f - Tr_{e\f} rho_e of the pairs its cut crosses.
 *
 * A shard's problem holds the regions it owns plus ghost regions (region_ghost), the other
 * endpoints of its crossing pairs, in the unsharded problem's relative order, with the pairs
 * that touch an owned region (explicit pairs) and the unsharded term placement (term_region)
 * restricted to owned regions.  Per iteration:
 *   lrh_halo_pass    region pass of the owned regions at the current (nu, zeta): Gibbs states
 *                    and partial traces, per-region values (asynchronous)
 *   lrh_halo_pack    copies the send items' pieces into the caller's device buffer
 *   (the caller moves the buffers between shards: NCCL, gloo, or a device copy)
 *   lrh_halo_unpack  stores the received pieces: ghost children's states, ghost parents' traces
 *   lrh_halo_update  the Alg. 2 update of every message (crossing pairs on both shards, from the
 *                    same inputs), theta recurrence
 * With the same L_hat (lrh_options.lhat > 0, the unsharded problem's beta Lambda_G / 2) and
 * launch shapes, every message of a shard is bit-identical to the same pair's message of the
 * unsharded run (lrh_step).  lrh_bound returns the shard's share of the sum (ghost regions count
 * zero); the caller adds the shards' shares.  lrh_step, lrh_evaluate, lrh_solve, lrh_vjp and
 * lrh_autotune return LRH_EUNSUPPORTED for problems with ghost regions. */
#define LRH_HALO_STATE 0   /* item id = region with a parent: its state rho (D x D complex)           */
#define LRH_HALO_TRACE 1   /* item id = pair e->f: the partial trace Tr_{e\f} rho_e (D_f x D_f complex) */
typedef struct {
    int32_t kind;          /* LRH_HALO_STATE or LRH_HALO_TRACE */
    int32_t id;            /* region or pair index of this problem */
} lrh_halo_item;

/* Host-only plan of a problem description (no device work; usable without a GPU): the pairs
 * (pair order; arrays of pair_cap entries, each may be NULL), their number, each term's region
 * (term_region[n_terms], may be NULL) and Lambda_G (may be NULL), exactly as lrh_create would
 * build them.  LRH_EINVAL if pair_cap is below the number of pairs and a pair array is given. */
int lrh_plan_poset(const lrh_problem_desc* desc, int64_t pair_cap, int32_t* pair_parent, int32_t* pair_child,
                   int64_t* n_pairs, int32_t* term_region, double* lambda_G);

/* Register the exchange of a problem with ghost regions: `send` lists the pieces this shard
 * sends (states of owned regions with a parent, traces of pairs with an owned parent), `recv`
 * the pieces it receives (states of ghost regions, traces of pairs with a ghost parent), each in
 * buffer order.  Every ghost region with a parent must be received exactly once, and every pair
 * with a ghost parent too (LRH_EINVAL otherwise, naming the item).  Returns the complex entries
 * per instance of the send and receive buffers (buffers are [n_instances][elems] complex64).
 * Synchronises. */
int lrh_halo_set(lrh_problem* p, int32_t n_send, const lrh_halo_item* send, int32_t n_recv,
                 const lrh_halo_item* recv, int64_t* send_elems, int64_t* recv_elems);
int lrh_halo_pass(lrh_problem* p);
/* send / recv: device buffers on the problem's device, 16-byte aligned, stream-ordered. */
int lrh_halo_pack(lrh_problem* p, void* send);
int lrh_halo_unpack(lrh_problem* p, const void* recv);
/* LRH_EINVAL unless lrh_halo_pass ran since the last update. */
int lrh_halo_update(lrh_problem* p);

#ifdef __cplusplus
}
#endif
#endif /* LRH_H */
