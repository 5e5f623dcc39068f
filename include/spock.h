/*
 * spock.h -- C ABI of libspock: the SPOCK method (preconditioned
 * Chambolle-Pock iteration accelerated by SuperMann with Anderson directions)
 * for scenario-tree risk-averse optimal control problems (RAOCPs) with AV@R
 * risk, on one NVIDIA B300 (sm_103a).
 *
 * Conventions for every call
 *  - Plain C types only. Host pointers are marked (host), device pointers
 *    (device); a device pointer must come from the CUDA runtime on the
 *    current device and be 16-byte aligned.
 *  - Every call returns an int status: SPOCK_OK (0), a positive warning, or a
 *    negative error. Errors leave the outputs unspecified but never abort the
 *    process and never trap the GPU. spock_status_str() names a status.
 *  - The library copies every input array it is given; the caller keeps
 *    ownership of its arrays. The library owns the device memory of a problem
 *    until spock_problem_destroy().
 *  - Calls on one problem are not thread-safe; different problems may be used
 *    from different host threads.
 *
 * Problem statement (Sec. 3 of the paper):
 *  - scenario tree (Sec. 3.2): n nodes in breadth-first order (stage-major,
 *    children of a node contiguous, all leaves at stage N and last), given by
 *    anc[] (anc[0] = -1) and prob[] = conditional probability of a node given
 *    its ancestor (prob[0] = 1, children probabilities of a node sum to 1);
 *  - dynamics (Eq. finite-horizon-evolution): x^c = A^c x^anc(c) + B^c u^anc(c)
 *    + c^c for every non-root node c, x^0 = x0;
 *  - costs (Sec. 3.2, "Quadratic-plus-linear costs"): edge cost
 *    x'Q^c x + u'R^c u + q^c'x + r^c'u on the ancestor's (x, u) for every
 *    non-root c, terminal cost x'Q_N^j x + q_N^j'x at every leaf j; Q, R, Q_N
 *    diagonal or full, linear terms optional;
 *  - constraints (Eq. constraints): optional box on x at every node (the
 *    root's box is applied to the fixed x0), optional box on u and optional
 *    Euclidean ball ||u||_2 <= r on u at every non-leaf node, and optional
 *    general rows Gx x + Gu u in a box at every non-leaf node and GN x in a
 *    box at every leaf;
 *  - risk (Sec. 3.3-3.4): AV@R_a over the children of every non-leaf node,
 *    a in [0, 1] per non-leaf node; the problem is the nested formulation
 *    Eq. original-problem, solved through its conic reformulation
 *    Eq. min-s0-v1 (Sec. 4).
 *
 * The preconditioning of Sec. 5.4 uses the diagonal entries of full weights
 * and scales every constraint row of a node, general rows included, by one
 * a = max{1, ||[Gx Sx^-1, Gu Su^-1]||_2}.
 *
 * Vector layout used by the operator-level calls (scaled variables, Sec. 4.3
 * "Sets" and Sec. 4.4 "Linear operator L"); first n_nl nodes are non-leaf:
 *   z   = [ s0 | x (n*nx) | u (n_nl*nu) | y (sum_i 2 n_i + 1) | tau (n-1) | s (n-1) ]
 *   eta = [ eta_y | eta_s (n_nl) | eta_c (n_nl*n_c) | eta_q ((n-1)(nx+nu+2))
 *         | eta_cN (n_l*n_cN) | eta_qN (n_l*(nx+2)) ]
 *   v   = [ z | eta ]  (n_v = n_z + n_eta elements)
 * with tau^c, s^c (c >= 1) at index c-1 of their arrays and constraint rows
 * [x box (nx)] [u box (nu)] [u ball (nu)] [general (n_g)] per non-leaf node,
 * [x box (nx)] [general (n_gN)] per leaf.
 */
#ifndef SPOCK_H
#define SPOCK_H

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define SPOCK_OK 0
#define SPOCK_MAXITER 1      /* warning: not converged within max_iters; outputs written */
#define SPOCK_PARTIAL 2      /* warning: only some plants were admitted (device memory) */
#define SPOCK_EINVAL -1      /* invalid argument (tree shape, sizes, probabilities, NULL) */
#define SPOCK_ENOMEM -2      /* device memory could not be allocated / admission refused */
#define SPOCK_ENOTPD -3      /* Cholesky of R~ = I + sum B'PB failed (not positive definite) */
#define SPOCK_EDEVICE -4     /* CUDA runtime error */
#define SPOCK_ETIMEOUT -5    /* a device-side wait (grid barrier) ran out of its time limit */
#define SPOCK_EUNSUPPORTED -6 /* sizes beyond the compiled limits (nx + nu <= 256, children <= 1024) */

#define SPOCK_MAX_NX 256     /* with nx + nu <= 256 */
#define SPOCK_MAX_NU 256

typedef struct spock_problem spock_problem;

/* Problem data (host arrays, row-major, float64). Sizes: n = n_nodes,
 * n_nl = non-leaf count, n_l = leaf count (derived from anc). */
typedef struct spock_problem_desc {
    int n_nodes;
    const int* anc;          /* [n] ancestor, anc[0] = -1 (Sec. 3.2) */
    const double* prob;      /* [n] conditional probability given the ancestor */
    int nx, nu;              /* state and input dimensions (Sec. 3.1) */
    const double* A;         /* [(n-1) nx nx]  A^c of node c at (c-1) */
    const double* B;         /* [(n-1) nx nu]  B^c */
    const double* c;         /* [(n-1) nx]     c^c, or NULL for zero */
    const double* Q;         /* [(n-1) nx]     diagonal of Q^c (edge cost on x^anc(c)) */
    const double* R;         /* [(n-1) nu]     diagonal of R^c (edge cost on u^anc(c)) */
    const double* QN;        /* [n_l nx]       diagonal of Q_N^j, leaves in node order */
    const double* x_lo;      /* [n nx] or NULL (no state box) */
    const double* x_hi;      /* [n nx] or NULL */
    const double* u_lo;      /* [n_nl nu] or NULL (no input box) */
    const double* u_hi;      /* [n_nl nu] or NULL */
    const double* u_ball;    /* [n_nl] ball radius on u, or NULL (no ball) */
    const double* avar;      /* [n_nl] AV@R level in [0, 1] (Sec. 3.3) */
    /* ---- optional parts of the problem statement; zero-initialise the struct
     *      (memset or = {0}) so that absent parts read as 0 / NULL ---------- */
    int weights_full;        /* 1: Q [(n-1) nx nx], R [(n-1) nu nu], QN [n_l nx nx] are full
                                symmetric positive definite matrices (Sec. 3.2); 0: diagonals
                                as above. L applies their upper Cholesky factors (SPOCK_ENOTPD
                                if one is not positive definite) */
    const double* q;         /* [(n-1) nx] linear edge cost q^c'x^anc(c), or NULL */
    const double* r;         /* [(n-1) nu] linear edge cost r^c'u^anc(c), or NULL */
    const double* qN;        /* [n_l nx]   linear terminal cost, or NULL. Linear terms enter
                                through the translation of the cost cones (Prop. 1 with
                                S = I): the weight must be positive definite where a linear
                                term is nonzero (SPOCK_EINVAL otherwise) */
    int n_g;                 /* general rows at every non-leaf node (Eq. constraints):
                                g_lo <= Gx x^i + Gu u^i <= g_hi, 0 <= n_g <= 256 */
    const double* Gx;        /* [n_g nx] (the same rows at every non-leaf node) */
    const double* Gu;        /* [n_g nu] */
    const double* g_lo;      /* [n_nl n_g] */
    const double* g_hi;      /* [n_nl n_g] */
    int n_gN;                /* general rows at every leaf: gN_lo <= GN x^j <= gN_hi, <= 256 */
    const double* GN;        /* [n_gN nx] */
    const double* gN_lo;     /* [n_l n_gN] */
    const double* gN_hi;     /* [n_l n_gN] */
    double l1;               /* lambda_0 >= 0: every edge cost gets the term
                                lambda_0 ||(x^anc, u^anc)||_1 (Prop. 2); 0: none. Solved through
                                auxiliaries theta^i, lambda^i per non-leaf node (shared by the
                                edge costs of its children, whose l1 terms are the same function of
                                (x^i, u^i)) appended to z, and the rows theta - sum lambda,
                                lambda - z, lambda + z in R_+ appended to eta. Single-problem
                                calls only: the batched and serving calls return
                                SPOCK_EUNSUPPORTED for such a problem */
    const double* tv;        /* [n_nl] radius r >= 0, or NULL. Non-NULL: the risk of every non-leaf
                                node is the worst expectation over the total-variation ball
                                {mu in the simplex : ||mu - p||_1 <= r} around its children's
                                probabilities (r = 0: the expectation; r >= 2: the maximum), a
                                conic risk with F != 0 (Sec. 3.3: nu >= |mu - p|, y^i of 3 n_i + 2
                                entries, S2^i = ker[E', -I, -I; F', 0, 0]); avar is then unused.
                                Single-problem calls only (as l1) */
    const double* soft_max;  /* [nx + nu] finite, or NULL. Non-NULL: every edge cost gets the
                                soft-constraint penalty ||max(0, (x^anc, u^anc) - soft_max)||^2
                                (the quadratic penalty after Prop. 2), through sigma^i >= ||theta^i||^2
                                (a translated second-order cone), theta^i >= 0 and
                                theta^i >= (x^i, u^i) - soft_max per non-leaf node (shared by its
                                children's edge costs) and tau^c - sigma^i in the children's cost
                                cones. Needs diagonal weights and l1 = 0 (SPOCK_EUNSUPPORTED
                                otherwise); single-problem calls only */
} spock_problem_desc;

typedef struct spock_sizes {
    int n, n_nonleaf, n_leaf, N, nx, nu, n_c, n_cN;
    long long n_z, n_eta, n_v;
    long long factor_bytes_fp64;   /* device bytes of the per-iteration factors, FP64 copy */
    long long factor_bytes_fp32;   /* same, FP32 copy */
    long long solve_bytes_fp64;    /* device bytes of the solve buffers of an FP64 solve (one
                                      allocation, made by the first solve in that precision) */
    long long solve_bytes_fp32;    /* same for FP32 */
    long long device_bytes;        /* device bytes the problem holds now (data, factors of
                                      both precisions, the solve buffers allocated so far) */
    long long device_peak_bytes;   /* the most it has held: the offline part's peak (its
                                      setup-only buffers included) or device_bytes */
} spock_sizes;

/* spock_problem_create: validate the tree and data, copy them to the device,
 * and run the offline part on the GPU in FP64 -- the preconditioning of
 * Sec. 5.4, Alg. 1 (projection on S1, offline) and ||L|| of Sec. 4.4 giving
 * alpha = 0.99/||L|| (Sec. 4.1 needs alpha ||L|| < 1). Also builds the FP32
 * copies of the factors. Errors: SPOCK_EINVAL (tree not breadth-first,
 * probabilities, sizes), SPOCK_EUNSUPPORTED, SPOCK_ENOTPD, SPOCK_ENOMEM,
 * SPOCK_EDEVICE. On error *out is NULL. */
int spock_problem_create(const spock_problem_desc* desc, spock_problem** out);
void spock_problem_destroy(spock_problem* p);

int spock_problem_sizes(const spock_problem* p, spock_sizes* out);

/* Step size alpha and ||L||. set_alpha overrides alpha (must satisfy
 * 0 < alpha ||L|| < 1, else SPOCK_EINVAL). */
int spock_problem_alpha(const spock_problem* p, double* alpha, double* normL);
int spock_problem_set_alpha(spock_problem* p, double alpha);

/* Scalings of Sec. 5.4 (host outputs): Sx[nx], Su[nu], SxN[nx]. */
int spock_problem_scalings(const spock_problem* p, double* Sx, double* Su, double* SxN);

/* FP64 output of Alg. 1 (host outputs, may be NULL): P [n nx nx], K [n_nl nu nx],
 * Rtilde [n_nl nu nu], Abar [(n-1) nx nx] (scaled problem). */
int spock_problem_factors(const spock_problem* p, double* P, double* K, double* Rtilde,
                          double* Abar);

/* Initial state used by the operator-level calls (host, unscaled, [nx]). */
int spock_problem_set_x0(spock_problem* p, const double* x0);

/* ---------------- operator-level calls (device pointers, async on stream) -----
 * precision: 64 (double vectors) or 32 (float vectors). stream: a cudaStream_t
 * or NULL for the default stream. */

/* One Chambolle-Pock step v_out = T(v_in) (Eq. chambolle-pock-operator) with
 * the problem's x0 and alpha: prox_{alpha f} of Eq. f (s0 - alpha, proj_S1 by
 * Alg. 2, proj_S2) and prox_{alpha g*} of Eq. g (Moreau, proj_S3 of
 * Eq. S3-def). v_in, v_out: (device) [n_v], must not overlap.
 * stats (host, may be NULL) receives 8 doubles of r = v_in - v_out:
 * [ max|r|, ||r_z||^2, ||r_eta||^2, <r_eta, L r_z>, 0, 0, 0, 0 ]. Blocking. */
int spock_op_T(spock_problem* p, int precision, const void* v_in, void* v_out, double* stats,
               void* stream);

/* One FP32 evaluation of T in the centred form (the map the centred FP32
 * iteration runs on, spock_solve_opts.recentre): out = T(c + delta) - c.
 * prox_f is affine (Alg. 2), so its part of the map is its linear part applied
 * to the increment in FP32, plus z+_c - z_c from one FP64 evaluation of T at c;
 * L acts on the increments; the prox of alpha g* (Moreau, proj_S3) is taken in
 * FP64 on c + the increment. Rounding is relative to the increments, not to c.
 * c (device) [n_v] FP64; delta, out (device) [n_v] FP32, distinct; stats as
 * for spock_op_T (of r = delta - out). Uses the problem's FP64 solve buffers
 * TV and VT and the centre buffers as scratch. Blocking. */
int spock_op_T_centred(spock_problem* p, const double* c, const float* delta, float* out, double* stats,
                       void* stream);

/* spock_op_T_noalloc: the same evaluation of T as spock_op_T, for callers that
 * cannot allocate device memory at the time of the call -- for example code
 * running under a memory pool or allocator it does not own, inside a
 * real-time loop where an allocation could block, or in a process whose
 * device memory is fully reserved by another framework. It calls no
 * cudaMalloc/cudaFree: all of its scratch (control block, barrier flags,
 * reduction partials, the sweep vectors and, when nx + nu <= 128, the sweep
 * mailboxes: 2 (n nx + n_nl nu) values, 2 n (nx + nu) mailbox entries of
 * 8 bytes (FP32) or 16 bytes (FP64), plus about 160 KB) comes from one
 * static device array of
 * SPOCK_NOALLOC_SCRATCH_BYTES, which every GPU that loads the library holds
 * until the process exits. Problems needing more return SPOCK_EUNSUPPORTED.
 * The first call on a device looks the array's address up on that device
 * (it must be the current device); make that first call before any stream
 * capture. Every call shares the array and resets what must start at zero;
 * calls that overlap on the GPU (other streams, other threads) race and must
 * be serialised by the caller. The paper has no counterpart of this call.
 * Arguments, layout and stats as for spock_op_T. Blocking. */
#define SPOCK_NOALLOC_SCRATCH_BYTES (8 << 20)
int spock_op_T_noalloc(spock_problem* p, int precision, const void* v_in, void* v_out,
                       double* stats, void* stream);

/* eta = L z (Sec. 4.4) and z = L* eta. (device) buffers of n_z / n_eta elements. */
int spock_op_L(spock_problem* p, int precision, const void* z, void* eta, void* stream);
int spock_op_Lt(spock_problem* p, int precision, const void* eta, void* z, void* stream);

/* ---------------- solve -------------------------------------------------------*/
typedef struct spock_solve_opts {
    int precision;        /* 64 or 32: arithmetic of the iteration (factors are FP64-built) */
    double tol;           /* stop when ||v - T(v)||_inf <= tol (Sec. 5.3, eps_rel = 0) */
    int max_iters;        /* outer iteration cap; SPOCK_MAXITER when reached */
    int max_backtracks;   /* cap on tau halvings per iteration (then v <- T(v)) */
    int method;           /* 0: SPOCK (Alg. 4 with Alg. 3, m = 3); 1: plain CP v <- T(v) */
    int warm_start;       /* 1: start from the problem's last iterate, 0: z = eta = 0 */
    int fp64_check;       /* 1 (FP32 only): finish with an FP64 residual check */
    int aa_mode;          /* Anderson least squares (Alg. 3): 0 the 3 x 3 normal equations
                             (Gram matrix accumulated in FP64, Cholesky; the default),
                             1 a QR factorisation of Y kept up to date as pairs enter and
                             leave (Givens rotations, Gram-Schmidt; Sec. 6.2), one more
                             pass over the vectors per iteration */
    double recentre;      /* FP32 only (spock_solve / spock_solve_device). 0: the iterate v
                             itself is held and iterated in FP32. > 0 (the default, 0.1):
                             centred FP32 iteration. An FP64 centre c is kept and the FP32
                             iteration runs on delta = v - c, i.e. on the map
                             delta -> T(c + delta) - c. Its linear parts act on the small
                             increments in FP32 and its projections are taken in FP64 about c.
                             Once the FP32 residual falls below recentre times the centre's
                             FP64 residual, the iterate moves into c (c += delta, delta = 0)
                             and the iteration restarts there (Anderson memory emptied).
                             The stopping test is the FP64 residual of the centre, so
                             res_inf = res_inf_fp64 is an FP64 figure. The iterate lives in
                             FP64: warm starts continue from the FP64 iterate, and
                             spock_get_iterate returns it in both precisions. Must be < 1. */
} spock_solve_opts;

typedef struct spock_info {
    int status;           /* SPOCK_OK, SPOCK_MAXITER or an error */
    int iters;            /* outer iterations k */
    int n_T;              /* evaluations of T */
    int n_K0, n_K1, n_K2, n_fallback;   /* accepted step kinds of Alg. 4 */
    int n_backtracks;     /* total tau halvings */
    double res_inf;       /* ||v - T(v)||_inf at exit, in the iteration precision (FP64 in
                             the centred FP32 iteration) */
    double res_inf_fp64;  /* same in FP64 (fp64_check), else = res_inf */
    double risk;          /* s^0 of T(v): the risk value (Sec. 4, Eq. min-s0-v1) */
    double device_ms;     /* device time of the solve (CUDA events): the solve kernel, and in
                             the centred FP32 iteration every segment with its re-centring */
    double phase_ms[7];   /* device time per phase seen by the first CTA, barrier waits
                             included: prep/S2, backward sweep, forward sweep + eta update,
                             T reductions, Anderson dots, direction pass, K2/backtrack passes */
    double counters[8];   /* SM cycles seen by the first thread of the first CTA: backward
                             sweep bulk-copy waits, mat-vecs, team reductions, other step
                             work; grid barriers, all-reductions; barrier and all-reduction
                             counts */
    /* FP64 exit check at the returned iterate v and its image T(v) (Sec. 5.3,
     * "Termination"; FP64 solves always, FP32 solves with fp64_check, else NaN):
     *   xi1    = ||(z - z+)/alpha - L*(eta - eta+)||_inf      (Eq. xi1k)
     *   xi2    = ||(eta - eta+)/alpha - L(z - z+)||_inf
     *   infeas = ||L z+ - proj_S3(L z+)||_inf                 (primal infeasibility)
     *   gap    = |<eta+, L z+> - sigma_S3(eta+)|               (complementarity gap,
     *            sigma_S3 the support function of S3 of Eq. S3-def) */
    double xi1, xi2, infeas, gap;
    int n_recentre;       /* centred FP32 iteration: centres taken (each one FP64 evaluation
                             of T, counted in n_T), else 0 */
    double kernel_ms;     /* device time of the iteration kernel's launches alone (CUDA
                             events around each; in the centred FP32 iteration the sum over
                             its FP32 segments), part of device_ms */
} spock_info;

void spock_solve_opts_default(spock_solve_opts* o);

/* Solve from host buffers (end-to-end: host->device copy of x0, solve,
 * device->host copy of the outputs, all inside the call). x0 (host) [nx],
 * unscaled; x_out (host) [n nx], u_out (host) [n_nl nu], unscaled, from T(v)
 * at exit; risk (host) scalar; info (host) may be NULL. Blocking. */
int spock_solve(spock_problem* p, const double* x0, const spock_solve_opts* opts,
                double* x_out, double* u_out, double* risk, spock_info* info);

/* Same with device buffers, enqueued on `stream` (blocking only for info):
 * x0 (device, double) [nx]; x_out, u_out (device, double) may be NULL. */
int spock_solve_device(spock_problem* p, const double* x0, const spock_solve_opts* opts,
                       double* x_out, double* u_out, void* stream, spock_info* info);

/* FP64 exit check of any iterate (Sec. 5.3): T(v) in FP64, then the
 * residual and the optimality measures of spock_info (xi1, xi2, infeas, gap)
 * plus the two terms of the gap. v (device) [n_v] in `precision` 32 or 64,
 * scaled variables (the layout above). Uses the problem's FP64 solve buffers
 * as scratch (allocated on first use): the current iterate kept for warm
 * starts is not touched. Blocking. */
typedef struct spock_check_info {
    double res_inf;       /* ||v - T(v)||_inf in FP64 */
    double xi1, xi2, infeas, gap;
    double eta_Lz;        /* <eta+, L z+> */
    double support;       /* sigma_S3(eta+) */
} spock_check_info;
int spock_check(spock_problem* p, int precision, const void* v, void* stream, spock_check_info* out);

/* Device copy of the current iterate v (after a solve) and a way to set it
 * (warm start). (device) buffers of n_v elements in the given precision. */
int spock_get_iterate(spock_problem* p, int precision, void* v_out, void* stream);
int spock_set_iterate(spock_problem* p, int precision, const void* v_in, void* stream);

/* ---------------- batched solves (many independent problems, one launch) -----
 * Many problems of different sizes (each created with spock_problem_create,
 * nx + nu <= 126) are solved together: one persistent launch in which every
 * CTA takes problems from a queue, largest first, and runs the whole iteration
 * of its problem (Sec. 5: T, Alg. 3, Alg. 4) with its barriers and reductions
 * inside the CTA. The device work of a solve (x0 upload, scaling, the launch,
 * unscaling, result download) is captured once into a CUDA graph and replayed.
 * The paper solves one problem per run; the batch is this library's addition. */
typedef struct spock_batch spock_batch;

typedef struct spock_batch_info {
    int status;           /* SPOCK_OK, SPOCK_MAXITER or SPOCK_ETIMEOUT for this problem */
    int iters;            /* outer iterations */
    int n_T;              /* evaluations of T */
    int tw;               /* warps per team of the problem's sweeps */
    double res_inf;       /* ||v - T(v)||_inf at exit, iteration precision */
    double risk;          /* s^0 of T(v) */
    double device_ms;     /* time the problem's CTA spent on it (SM clock) */
    double xi1, xi2, infeas, gap;   /* FP64 exit check as in spock_info, when opts->fp64_check
                                       is set (computed after the launch, outside total_ms),
                                       else NaN */
} spock_batch_info;

/* Bundle `count` problems (not copied: they must outlive the batch and must not
 * be solved on their own while the batch is in use, since the batch uses their
 * solve buffers) for iteration in `precision` (32 or 64). The batch keeps each
 * problem's iterate between solves (warm start). EUNSUPPORTED if some problem
 * has nx + nu > 126. */
int spock_batch_create(spock_problem* const* problems, int count, int precision, spock_batch** out);
void spock_batch_destroy(spock_batch* b);

/* Totals of the packed host arrays of spock_batch_solve: x0 [sum nx],
 * x_out [sum n nx], u_out [sum n_nl nu] (problem after problem). */
int spock_batch_sizes(const spock_batch* b, long long* x0_total, long long* x_total, long long* u_total);

/* Warps per team of each problem's sweeps: tw[i] in {1, 2, 4, 8} with
 * 64 tw[i] >= nx + nu; NULL restores the default. */
int spock_batch_set_tw(spock_batch* b, const int* tw);

/* Autotuner: times `iters` plain CP iterations of every problem for each
 * admissible warps-per-team choice, with and without streaming the factors
 * through shared memory, and keeps the fastest per problem. Leaves every
 * iterate at zero. tw_out [count] (may be NULL) receives the choices. */
int spock_batch_autotune(spock_batch* b, int iters, int* tw_out);

/* Solve every problem. x0 (host) packed [sum nx], unscaled; opts as for
 * spock_solve (precision must equal the batch's; fp64_check = 1 adds the FP64
 * exit check of every problem's final iterate to info, after the launch);
 * warm_start = 1 starts each problem from its last iterate. x_out, u_out
 * (host, packed, may be NULL), risk (host) [count] (may be NULL), info (host)
 * [count] (may be NULL). total_ms (may be NULL) receives the device time of
 * the whole replay (copies included). Blocking. Returns SPOCK_OK if every
 * problem converged, SPOCK_MAXITER if some did not, or the first error. */
int spock_batch_solve(spock_batch* b, const double* x0, const spock_solve_opts* opts, double* x_out,
                      double* u_out, double* risk, spock_batch_info* info, double* total_ms);

/* ---------------- serving (MPC requests, continuous batching) ----------------
 * Plants (problems) stay resident on the device with their factors and their
 * last iterate. Requests (plant, x0) are published into a ring in mapped host
 * memory; a persistent launch whose CTAs claim requests as they appear runs
 * each one alone in a CTA, so requests that arrive while others are on the GPU
 * start as soon as a CTA frees up, and a result does not depend on the other
 * requests in flight. Requests of one plant run one after the other (they share
 * the plant's iterate). The launch leaves after 1 s without requests and is
 * restarted by the next call. The paper has no serving layer; this is the
 * library's addition. Plants need nx <= 64, nu <= 64, nx + nu <= 126. */
typedef struct spock_server spock_server;

typedef struct spock_serve_result {
    long long id;         /* as returned by spock_server_submit */
    int plant;
    int status;           /* SPOCK_OK, SPOCK_MAXITER or SPOCK_ETIMEOUT */
    int iters;
    int n_T;
    double res_inf;       /* ||v - T(v)||_inf at exit, iteration precision */
    double risk;          /* s^0 of T(v) */
    double u0[64];        /* first control u^0 (unscaled), nu entries */
    double device_ms;     /* time on the device from claim to result */
    double latency_ms;    /* host time from submission to the poll that saw the result */
} spock_serve_result;

/* Admit plants in the given order while their solve buffers
 * (spock_sizes.solve_bytes_fp32/_fp64) fit in the admission budget:
 * mem_budget bytes if mem_budget > 0 (clamped to the free device memory less
 * 256 MB), else the free device memory less 256 MB (plants whose buffers
 * already exist cost nothing);
 * *admitted (may be NULL) = how many. opts as for spock_solve (precision must
 * equal `precision`; fp64_check ignored); ring_slots >= 1 bounds the requests
 * on the device at once. Returns SPOCK_PARTIAL if some plants were refused,
 * SPOCK_ENOMEM if none fit. The plants must outlive the server and not be
 * solved on their own meanwhile. */
int spock_server_create(spock_problem* const* plants, int count, int precision, const spock_solve_opts* opts,
                        int ring_slots, long long mem_budget, spock_server** out, int* admitted);

/* Queue a request: x0 (host) [nx of the plant], unscaled; warm_start = 1
 * starts from the plant's last iterate. *id_out (may be NULL) = request id.
 * A request for a plant that is not admitted (refused at creation or evicted)
 * retries its admission against the room left at that moment (the budget
 * less what admitted plants were charged, never more than the free device
 * memory less 256 MB) and gets SPOCK_ENOMEM if it still does not fit.
 * Non-blocking (an admission allocates the plant's solve buffers). */
int spock_server_submit(spock_server* s, int plant, const double* x0, int warm_start, long long* id_out);

/* Collect up to max_out finished requests into out (host) and hand waiting
 * requests to the device; *n_out = how many were collected. Non-blocking. */
int spock_server_poll(spock_server* s, spock_serve_result* out, int max_out, int* n_out);

/* Requests submitted and not yet collected by spock_server_poll. */
long long spock_server_outstanding(const spock_server* s);

/* Release a plant: its solve buffers (and with them its warm-start iterate)
 * are freed and their bytes return to the admission budget, so a request for
 * a plant refused earlier can be admitted. The plant must have no request
 * submitted and not collected (SPOCK_EINVAL otherwise). The memory itself is
 * freed once the persistent launch is idle and has left (at a later poll or
 * at spock_server_destroy); with the default budget (free memory) it counts
 * for admission from then on. A later request for the plant re-admits it
 * (cold iterate if its buffers were freed). */
int spock_server_evict(spock_server* s, int plant);

/* 1 if the plant is admitted (its buffers resident for the server), 0 if not,
 * SPOCK_EINVAL for a bad handle or index. */
int spock_server_admitted(const spock_server* s, int plant);

/* Stop the persistent launch (after the requests in flight) and free. */
void spock_server_destroy(spock_server* s);

const char* spock_status_str(int status);
int spock_version(void);

/* Fault injection for tests of the failure path; the paper has no counterpart.
 * Every later single-problem launch (spock_solve*, spock_op_T, spock_check)
 * makes its grid barriers wait for `phantom_ctas` (0..4) CTAs beyond the ones
 * it launches, and gives up one barrier wait after wait_limit_s seconds
 * (0: the default 2 s; at most 10 s). With phantom_ctas > 0 the first barrier
 * wait therefore runs out, the launch records the timeout, every CTA leaves
 * after its bulk copies have landed, and the call returns SPOCK_ETIMEOUT; no
 * GPU fault is involved and the CUDA context stays usable. (0, 0) restores
 * normal launches. Process-wide, not thread-safe. SPOCK_EINVAL for values out
 * of range. */
int spock_debug_wait_fault(int phantom_ctas, double wait_limit_s);

/* Bounds-checked build (libspock_checked.so, compiled with -DSPOCK_CHECKED;
 * a stand-in for a memory sanitizer where none is available): the
 * single-problem iteration kernel checks the indices it derives
 * from the tree -- children ranges, segment nodes, mailbox slots, the factor
 * blocks its bulk copies read -- before use. A failed check skips the access,
 * ends the launch (SPOCK_EDEVICE) and is reported here: the site of the last
 * failed check, 0 if none failed since load; -1 in the regular library.
 * Not a call of the paper. */
int spock_debug_last_check(void);

#ifdef __cplusplus
}
#endif
#endif /* SPOCK_H */
