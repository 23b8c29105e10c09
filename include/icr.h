/*
 * icr.h - C ABI of libicr, the GB300 (sm_103a) implementation of the fast
 * constraint-matrix update for implicit contact resolution
 * ("An efficient implicit constraint resolution scheme for interactive FE
 * simulations", arXiv 2306.06946).
 *
 * Problem statement (Sec. 3 and Sec. 5 of the paper).  A deformable body with
 * n DOFs has the SPD system matrix A = M + h B + h^2 K (Sec. 3.1, Eq.
 * "dynamic equation soft").  m contacts each carry a proximity point
 * p_a = G(q) given by barycentric weights on 4 nodes, so H = dG/dq is 3m x n
 * (Eq. "geometrical mapping"), and a 3x3 direction block C_a whose rows are
 * the normal n and the tangents t1, t2 (Eq. "jacobian directions").  With
 * J = C H (Eq. "isolate directions") the Delassus operator is
 * W = J A^-1 J^T = C W_H C^T, W_H = H A^-1 H^T (Eq. "schur complemnt
 * reformulated").  W_H is built once per time step; every Newton iteration of
 * Alg. 3 re-forms W from new directions, solves the frictional contact problem
 * by projected Gauss-Seidel (Eq. "PGS") and moves the proximity points by
 * W_H C^T lambda (Eq. "recursive motion correction 7").  The corrective motion
 * dq = A^-1 H^T sum_k C_k^T lambda_k (Eq. "recursive motion correction 3") is
 * applied once at the end of the step.
 *
 * Units: the library works with lambda~ = h^2 lambda, so delta = delta_free +
 * W lambda~, dq = A^-1 J^T lambda~ is a position increment and the physical
 * contact force is lambda~ / h^2.
 *
 * Ordering: the system is given through its supernodal factor A = L D L^T in
 * the factor's DOF order, DOF = 3 * node + axis; supernodes hold whole nodes
 * (their column ranges start and end on multiples of 3).  Node ids passed to
 * icr_set_mapping are in that same order.
 *
 * Ownership: every set/update call copies what it is given; the caller keeps
 * its buffers.  The scene owns all device state; nothing returned aliases it.
 *
 * Streams: all work of a scene is enqueued on the context's stream.  Calls
 * that write to host memory (icr_get, non-NULL *_out host pointers, stats)
 * synchronise that stream before returning; the others return once the work
 * is enqueued.
 *
 * Threads: a context and its scenes are used by one host thread at a time;
 * different contexts may be used from different threads.
 *
 * Errors: every call returns ICR_OK or one of the codes below and leaves a
 * message for icr_last_error() (thread-local).
 */
#ifndef ICR_H_
#define ICR_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum icr_status {
  ICR_OK = 0,
  ICR_EINVAL = 1,    /* bad argument: shape, range, NaN, non-orthonormal C, bad weights */
  ICR_ENOTSPD = 2,   /* a pivot D_i is <= 0 or not finite */
  ICR_ESTATE = 3,    /* calls out of order (e.g. icr_update_W before icr_build_WH) */
  ICR_ENOMEM = 4,    /* device allocation failed or the context's HBM budget is exceeded */
  ICR_ENOCONV = 5,   /* non-fatal: PGS used all sweeps with eps above a positive tol */
  ICR_ETIMEOUT = 6,  /* a bounded device-side wait gave up */
  ICR_ECUDA = 7      /* a CUDA runtime call failed */
};

enum icr_precision {
  ICR_FP32 = 0,      /* L, X, W_H, W, the tangent frames and the PGS sweeps in FP32; gaps, p and u
                        accumulated in FP64 */
  ICR_FP64 = 1       /* everything in FP64 */
};

typedef struct icr_ctx icr_ctx;       /* one device + one CUDA stream + an HBM budget */
typedef struct icr_scene icr_scene;   /* one deformable body with its contacts */

/* How the contraction W_H = Y^T Y (Y = D^-1/2 L^-1 H^T) is computed in an FP32
 * scene.  FP64 scenes always use FP64 SIMT arithmetic.  In the three
 * tensor-core modes the forward solve of the wide fronts also runs on the
 * tensor cores, always in 3xTF32, in the etree levels icr_autotune assigns
 * them; tensor-core partial sums are added into FP32 registers every 128 K. */
enum icr_contraction {
  ICR_CONTRACT_AUTO = 0,    /* FP32 scenes: ICR_CONTRACT_TF32X3 */
  ICR_CONTRACT_SIMT = 1,    /* FP32 CUDA cores for the contraction and the forward solve */
  ICR_CONTRACT_TF32X3 = 2,  /* tensor cores, each operand split into a TF32 part and a TF32 remainder,
                               three products (W_H within 3e-6 of FP64 at 60k DOF, CUDA cores 3e-7) */
  ICR_CONTRACT_TF32 = 3,    /* tensor cores, TF32 operands, FP32 accumulation */
  ICR_CONTRACT_BF16 = 4     /* tensor cores, BF16 operands, FP32 accumulation */
};

/* Operand precision of W = C W_H C^T (Alg. 3 step 2) in an FP32 scene; the
 * products are accumulated in FP32 in every mode.  FP64 scenes ignore it. */
enum icr_w_update {
  ICR_W_FP32 = 0,   /* C and W_H as stored (FP32) */
  ICR_W_TF32 = 1,   /* C and W_H rounded to TF32 (10-bit mantissa) before the products */
  ICR_W_BF16 = 2    /* W_H read from a BF16 copy written when W_H is formed (half the bytes per
                       update), C rounded to BF16 */
};

typedef struct icr_params {
  int32_t precision;     /* enum icr_precision */
  int32_t n_sweeps;      /* PGS sweep cap (>= 0) */
  double tol;            /* PGS stop when eps <= tol (tol > 0); a sweep without change always stops */
  int32_t contraction;   /* enum icr_contraction */
  int32_t warm_start;    /* 1: the first PGS of a time step (Newton iteration 1) starts from the
                            previous step's iteration-1 lambda~ (zero before the first step),
                            Newton iterations 2..k start from 0 (incremental reading of Alg. 3);
                            0: every PGS starts from 0.  Read by icr_step / icr_step_capture. */
  int32_t w_update;      /* enum icr_w_update */
  double newton_tol;     /* >= 0.  0: icr_step runs all n_newton iterations.  > 0: after the proximity
                            update of iteration k the step linearises for iteration k + 1 and
                            evaluates, in FP64, the normal complementarity residual of a zero increment
                            at those gaps, max over contacts of max(0, -delta_n); when it is at most
                            newton_tol the next solve has nothing to correct and the Newton loop ends
                            (the remaining iterations' kernels return at once; the corrective motion
                            runs).  icr_newton_iterations reports the iterations run. */
} icr_params;

typedef struct icr_pgs_stats {
  int32_t sweeps;       /* sweeps run */
  int32_t n_separated;  /* contacts with lambda_n = 0 */
  int32_t n_stick;      /* contacts strictly inside the friction cone */
  int32_t n_slip;       /* contacts on the cone (||lambda_t|| >= mu lambda_n (1 - rel), rel = 1e-9 in FP64
                           scenes and 1e-5 in FP32 scenes; a loaded frictionless contact counts here) */
  double eps;           /* ||lambda^i - lambda^(i-1)|| / ||lambda^i|| of the last sweep (Alg. 1) */
  double res_normal;    /* FP64 max |min(delta_n, lambda_n)| at the end */
  double res_cone;      /* FP64 max(0, ||lambda_t|| - mu lambda_n) */
  double res_stick;     /* FP64 max ||delta_t|| over sticking contacts */
  double res_slip;      /* FP64 max misalignment of delta_t against -lambda_t over slipping contacts with
                           lambda_t != 0 (with mu lambda_n = 0 the sliding is free) */
  int32_t sweeps_s_only;  /* sweeps that visited only the blocks of contacts that may change (the
                             others provably keep lambda~ = 0; see icr_solve_friction) */
  int32_t deferred_folds; /* folds of those sweeps' changes into the other contacts' residuals */
  int32_t rechecks;       /* rechecks of the other contacts' normal residuals when the bound ran out */
  int32_t joins;          /* rechecks after which the blocks of contacts that may change joined S */
} icr_pgs_stats;

enum icr_field {
  ICR_FIELD_WH = 0,        /* (3m x 3m) double, row-major, symmetric */
  ICR_FIELD_W = 1,         /* (3m x 3m) double */
  ICR_FIELD_LAMBDA = 2,    /* (3m) double, lambda~ of the last solve */
  ICR_FIELD_P = 3,         /* (m x 3) double, proximity positions */
  ICR_FIELD_DELTA = 4,     /* (3m) double, gaps the next solve starts from */
  ICR_FIELD_C = 5,         /* (m x 3 x 3) double, direction blocks, rows n, t1, t2 */
  ICR_FIELD_MU = 6,        /* (m) double, friction coefficients */
  ICR_FIELD_U = 7,         /* (3m) double, accumulated sum_k C_k^T lambda~_k */
  ICR_FIELD_REACH_PTR = 8, /* (nsuper + 1) int32, CSR offsets of the reached contacts */
  ICR_FIELD_REACH_IDX = 9, /* (reach_ptr[nsuper]) int32, ascending contact ids per supernode */
  ICR_FIELD_DQ = 10,       /* (n) double, the last corrective motion */
  ICR_FIELD_LAMBDA0 = 11   /* (3m) double, lambda~ of Newton iteration 1 of the last warm-started
                              device-resident step (the next step's warm start; zero before) */
};

/* Thread-local text of the last error (never NULL). */
const char* icr_last_error(void);

/* Context on CUDA device `device`.  `cuda_stream` is a cudaStream_t owned by
 * the caller (NULL = the legacy default stream).  `hbm_budget_bytes` caps the
 * device memory all scenes of the context may hold (0 = no cap); an
 * allocation past it fails with ICR_ENOMEM. */
int icr_ctx_create(icr_ctx** out, int device, void* cuda_stream, uint64_t hbm_budget_bytes);
int icr_ctx_destroy(icr_ctx* ctx);
/* Device bytes currently held by the context's scenes. */
int icr_ctx_bytes_in_use(const icr_ctx* ctx, uint64_t* out);

/* Bound of the tensor-core kernels' pipeline waits (the shared-memory ring
 * and the TMEM hand-offs between the MMA-issuing thread and the warps that
 * read the accumulators), in ns of the GPU's global timer; 1 s by default.
 * A wait that runs out (or sees the other side give up) ends the CTA's work:
 * bulk copies in flight are allowed to land and every issued MMA to complete
 * (each of these waits bounded by 1 s) before TMEM is freed, the scene's
 * device error word is set, and the next synchronising call of that scene
 * returns ICR_ETIMEOUT (its W_H is then incomplete; the next icr_build_WH
 * forms it again).  0 makes every pipeline wait a single non-blocking poll:
 * failure injection for tests of that path.  Kernels read the value when they
 * are launched (a captured step graph keeps the value of its capture). */
int icr_ctx_set_wait_limit(icr_ctx* ctx, uint64_t pipeline_wait_ns);

/* Failure injection: the device allocation after the next `after` ones made
 * for the context's scenes fails with ICR_ENOMEM (once; -1 switches it off).
 * A set call that fails part way leaves the scene without what it was
 * replacing (icr_set_system: no system; icr_set_mapping: no mapping; the
 * obstacle calls: no obstacle), so later calls return ICR_ESTATE until it is
 * set again. */
int icr_ctx_inject_alloc_failure(icr_ctx* ctx, int64_t after);

int icr_scene_create(icr_ctx* ctx, icr_scene** out, const icr_params* params);
int icr_scene_destroy(icr_scene* scene);
int icr_set_params(icr_scene* scene, const icr_params* params);

/* The system, through its supernodal factor A = L D L^T (Sec. 3.1, Eq.
 * "dynamic equation soft"; the factor plays the role of the preconditioner
 * the paper's results use, Sec. 6).  Host arrays:
 *   super_ptr    (nsuper+1) int32: supernode s owns DOF columns [super_ptr[s], super_ptr[s+1]),
 *                 increasing, multiples of 3, super_ptr[nsuper] = n;
 *   rowpat_ptr   (nsuper+1) int64 offsets into rowpat;
 *   rowpat       int32 below-diagonal rows R_s of each supernode, ascending, each >= super_ptr[s+1], < n;
 *   val_ptr      (nsuper+1) int64 offsets into Lpanels; panel s has (w+r) * w entries;
 *   Lpanels      double, panel s column-major (w + r) x w: rows 0..w-1 the unit lower diagonal
 *                 block (diagonal and upper part ignored), rows w..w+r-1 L[R_s, cols(s)];
 *   D            (n) double pivots, each finite and > 0 (else ICR_ENOTSPD);
 *   etree_parent (nsuper) int32 parent supernode (> s) or -1: the supernode owning min(R_s);
 *                 R_s minus the columns of the parent must lie in the parent's R.
 * Replaces any previous system and invalidates the mapping and W_H. */
int icr_set_system(icr_scene* scene, int32_t n, int32_t nsuper, const int32_t* super_ptr,
                   const int64_t* rowpat_ptr, const int32_t* rowpat, const int64_t* val_ptr,
                   const double* Lpanels, const double* D, const int32_t* etree_parent);

/* The geometric mapping H = dG/dq for barycentric proximity points
 * (Eq. "geometrical mapping"; Eq. "isolate directions" keeps it apart from
 * the directions).  nodes (m x 4) int32 node ids in factor order, bary
 * (m x 4) double weights, each >= 0 and summing to 1 within 1e-12.
 * m = 0 is allowed.  Resets lambda~ (and its warm start), mu, the directions,
 * the gaps, u and the proximity positions to 0. */
int icr_set_mapping(icr_scene* scene, int32_t m, const int32_t* nodes, const double* bary);

/* Proximity positions p (m x 3 double) after the free motion: the start of the
 * recursion p_0 (Alg. 3 step 4 updates it).  The scene keeps a device copy of
 * p_0 for icr_reset_proximity. */
int icr_set_proximity(icr_scene* scene, const double* p);
/* Start a time step again from the stored p_0: p <- p_0 and u <- 0, on the
 * device (no host transfer). */
int icr_reset_proximity(icr_scene* scene);

/* Directions and gaps for the next Newton iteration (Alg. 3 step 1).
 * C (m x 3 x 3 double, row-major blocks with rows n, t1, t2, each orthonormal
 * within 1e-6), delta (3m double) the gaps at the current proximity positions,
 * mu (m double, >= 0) or NULL to keep the previous coefficients. */
int icr_update_directions(icr_scene* scene, const double* C, const double* delta, const double* mu);

/* Device-side linearisation (Alg. 3 step 1 for two obstacle kinds): computes C
 * and delta from the current proximity positions without a host round trip.
 * Tangent frame: e_a = the axis with the smallest |n_a| (lowest index on ties),
 * t1 = normalize(n x e_a), t2 = n x t1.
 *   plane:  normals (n_iters x m x 3 double) unit normals for iteration k,
 *           anchors (m x 3): delta = C (p - anchor);
 *   sphere: centre (3), radius, anchors (m x 3): n = (p - c)/|p - c|,
 *           delta = (|p - c| - radius, t1.(p - anchor), t2.(p - anchor)). */
int icr_set_obstacle_plane(icr_scene* scene, int32_t n_iters, const double* normals, const double* anchors);
int icr_set_obstacle_sphere(icr_scene* scene, const double* center, double radius, const double* anchors);
/* Several sphere tools: spheres is n_spheres x 4 (centre x, y, z, radius > 0),
 * contact_sphere (m int32, each in [0, n_spheres)) names the tool each contact
 * touches, anchors as for one sphere.  icr_set_obstacle_sphere is the case
 * n_spheres = 1.  Copies its inputs; ICR_EINVAL on a bad radius or index. */
int icr_set_obstacle_spheres(icr_scene* scene, int32_t n_spheres, const double* spheres,
                             const int32_t* contact_sphere, const double* anchors);
/* A time step's inputs in one call: the same as icr_set_mapping(m, nodes,
 * bary), icr_set_proximity(p0), icr_set_obstacle_spheres(n_spheres, spheres,
 * contact_sphere, anchors) and icr_set_field(ICR_FIELD_MU, mu), with the same
 * checks and errors.  When the scene already holds m contacts and n_spheres
 * spheres, the inputs travel in one host-to-device copy through a pinned
 * staging buffer of the scene (two slots; a slot is reused only after its
 * previous copy has completed) and one kernel resets the contact state, so a
 * captured step graph stays valid; otherwise it makes the four calls.  The
 * host arrays may be released when the call returns. */
int icr_set_step_inputs(icr_scene* scene, int32_t m, const int32_t* nodes, const double* bary, const double* p0,
                        const double* mu, int32_t n_spheres, const double* spheres, const int32_t* contact_sphere,
                        const double* anchors);
int icr_linearize(icr_scene* scene, int32_t k);

/* W_H = H A^-1 H^T = X^T D^-1 X with X = L^-1 H^T (Eq. "schur complemnt
 * reformulated"): the symbolic reach of H^T in the elimination tree, the
 * multi-RHS supernodal forward solve, the FP64 pivot scaling and the
 * contraction.  Needs icr_set_system and icr_set_mapping. */
int icr_build_WH(icr_scene* scene);

/* W = C W_H C^T (Alg. 3 step 2).  Needs icr_build_WH and directions. */
int icr_update_W(icr_scene* scene);

/* Projected Gauss-Seidel on delta = delta_free + W lambda~ (Eq. "PGS", Alg. 3
 * step 3): contacts in ascending order; local rule: lambda_n <- max(0,
 * lambda_n - r_n / W_nn); the tangential residual is updated with the change
 * of lambda_n; lambda_t <- lambda_t - r_t / w_t with w_t = (W_t1t1 + W_t2t2)/2;
 * lambda_t is projected on the disc ||lambda_t|| <= mu lambda_n.
 * The solve stops after n_sweeps, when eps <= tol (tol > 0), or after a sweep
 * that changed no lambda~ (a fixed point: every later sweep would repeat it).
 * A contact with lambda~ = 0 and r_n >= 0 is left unchanged by the local rule,
 * so a sweep passes over it; once every residual is complete, the contacts
 * that may change (S, in blocks of 32, FP64 16) are swept alone while the sum
 * of |changes| since the bound's base stays below min r_n / max |W[n, j]|
 * over the others, the maximum over the columns j of S's blocks (their r_n
 * then stays non-negative).  When it runs out, the
 * others' normal residuals are formed with the deferred changes: all positive,
 * the bound starts again from there; else the changes reach the others'
 * residuals in one deferred fold and full sweeps resume.  The iterate is that
 * of full sweeps, up to the rounding of the residuals.
 * warm_start = 0 starts from lambda~ = 0, 1 from the last solve's lambda~.
 * stats (may be NULL) receives the sweep count, eps and FP64 residuals (this
 * synchronises).  Returns ICR_ENOCONV (non-fatal) when tol > 0 and eps > tol
 * after n_sweeps; the stats then say why. */
int icr_solve_friction(icr_scene* scene, int warm_start, icr_pgs_stats* stats);

/* p += W_H C^T lambda~ (Alg. 3 step 4, Eq. "recursive motion correction 7")
 * and u += C^T lambda~.  dp_out (3m double, host) receives the increment when
 * not NULL. */
int icr_update_proximity(icr_scene* scene, double* dp_out);

/* dq = A^-1 H^T u = L^-T D^-1 X u (Eq. "recursive motion correction 3"),
 * u = sum_k C_k^T lambda~_k.  dq_out (n double, host) may be NULL.  reset = 1
 * clears u afterwards (start of the next time step). */
int icr_correct_motion(icr_scene* scene, double* dq_out, int reset);

/* One time step of the fast scheme (Alg. 3) enqueued entirely on the device,
 * with directions from the scene's obstacle (icr_linearize): p <- p_0, u <- 0,
 * icr_build_WH, then n_newton x (icr_linearize(k), icr_update_W,
 * icr_solve_friction (from lambda~ = 0, or warm-started in iteration 1 per
 * icr_params.warm_start), icr_update_proximity), then
 * icr_correct_motion without a host copy (dq, p, lambda~ stay on the device).
 * Needs a system, a mapping, p_0 and an obstacle; returns once the work is
 * enqueued. */
int icr_step(icr_scene* scene, int32_t n_newton);
/* Newton iterations the last device-resident step (icr_step or a launch of
 * the captured step) ran: n_newton, or fewer when newton_tol ended the loop.
 * Synchronises. */
int icr_newton_iterations(icr_scene* scene, int32_t* out);
/* Capture icr_step(scene, n_newton) into a CUDA graph owned by the scene (one
 * plain step runs first so that every kernel is set up; icr_autotune runs
 * first when the scene is not tuned).  The context's stream must not be the
 * legacy default stream (ICR_EINVAL).  The graph reads the scene's device
 * buffers, so new inputs of the same shape (icr_set_mapping with the same
 * contact count, icr_set_proximity, the obstacle, icr_set_field) are stepped
 * by launching it again. */
int icr_step_capture(icr_scene* scene, int32_t n_newton);
/* Autotuner of the forward solve X = L^-1 H^T (the multi-RHS supernodal solve
 * of Eq. "schur complemnt reformulated").  For every elimination-tree level it
 * times the level's front products with three tile shapes: CUDA-core tiles of
 * 64 front rows x 96 columns, CUDA-core tiles of 32 rows x 96 columns (short
 * fronts), and 128 x 128 tcgen05 tiles (3xTF32, for fronts at least 64 wide
 * with 64 columns; FP32 scenes outside the SIMT contraction mode), on the
 * scene's current mapping, and keeps the fastest (the tensor cores must win by
 * 3 % over the faster CUDA-core tile).  Synchronises; runs several W_H builds
 * (W_H is left formed).  Needs a system and a mapping (ICR_ESTATE); not while
 * the stream is being captured (ICR_ESTATE).  tc_levels (may be NULL) receives
 * the number of levels on the tensor cores.  Until it runs, every level with
 * a front at least 64 wide uses the tensor cores and the others 64-row tiles;
 * icr_set_mapping and a change of contraction mode mark the scene untuned.
 * Each level's time is the median of 5 builds per tile shape, the shapes
 * alternating; level_ms (may be NULL when max_levels = 0) receives, for the
 * first max_levels levels (leaves first), the 64-row, the 32-row and the
 * tensor-core time in ms (the 64-row time again where the tensor cores do not
 * apply). */
int icr_autotune(icr_scene* scene, int32_t* tc_levels, double* level_ms, int32_t max_levels);
/* Fix the forward-solve plan instead of tuning it: for every etree level
 * (n_levels = icr_forward_levels, leaves first) 0 puts the level's fronts on
 * 64-row CUDA-core tiles, 1 its wide fronts on the tensor cores (where they
 * qualify, FP32 scenes outside the SIMT contraction mode; the others on 64-row
 * tiles), 2 on 32-row CUDA-core tiles.  Marks the scene tuned.  Needs a
 * system (ICR_ESTATE); ICR_EINVAL on a wrong count or a value above 2. */
int icr_set_forward_plan(icr_scene* scene, const uint8_t* tc_levels, int32_t n_levels);
int icr_forward_levels(icr_scene* scene, int32_t* n_levels);
/* Launch the captured step on the context's stream.  ICR_ESTATE without a
 * captured step, without a mapping and an obstacle, or when the graph is stale:
 * a buffer was reallocated, or the contact count, the obstacle kind or the
 * parameters differ from the capture (capture again). */
int icr_step_launch(icr_scene* scene);
/* Wait until the context's stream has finished the scene's work. */
int icr_sync(icr_scene* scene);

/* Continuous batching of time steps over resident scenes (a request loop).
 * Every scene must have a captured step (icr_step_capture) and live on one
 * device.  Request r asks for one step of scene req_scene[r] at time
 * req_arrival_s[r] (seconds from the call, non-decreasing).  The loop replays
 * the schedule in real time with n_slots concurrent streams: an arrived
 * request starts on a free slot as soon as its scene has no step in flight, so
 * requests that arrive while others run on the GPU overlap with them.
 * latency_s[r] receives arrival-to-completion seconds, *makespan_s (may be
 * NULL) the time until the last completion.  ICR_ETIMEOUT after timeout_s.
 * Slots only overlap on the GPU when the process has as many hardware work
 * queues (environment variable CUDA_DEVICE_MAX_CONNECTIONS, read when CUDA
 * starts; 8 by default): streams that share a queue run one after another. */
int icr_serve(icr_scene* const* scenes, int32_t n_scenes, const int32_t* req_scene, const double* req_arrival_s,
              int32_t n_req, int32_t n_slots, double timeout_s, double* latency_s, double* makespan_s);
/* icr_serve with admission under the HBM budget of each scene's context.
 * Scenes may be evicted (icr_scene_evict) when the call starts.  A request for
 * an evicted scene readmits it (icr_scene_readmit) before it starts; while the
 * context's budget is short, the least recently used resident scenes of that
 * context with no step in flight are evicted first.  A scene that does not fit
 * even then waits while other steps of its context are in flight and is
 * rejected (latency_s = -1) when none are.  stats (may be NULL) receives the
 * evictions, readmissions and rejections and the seconds spent admitting.
 * Eviction frees device memory (cudaFree), which waits for the device's work in
 * flight: admissions stall the loop while they run. */
typedef struct icr_serve_stats {
  int32_t evictions;
  int32_t readmissions;
  int32_t rejected;
  double admit_s;
} icr_serve_stats;
int icr_serve_ex(icr_scene* const* scenes, int32_t n_scenes, const int32_t* req_scene, const double* req_arrival_s,
                 int32_t n_req, int32_t n_slots, double timeout_s, double* latency_s, double* makespan_s,
                 icr_serve_stats* stats);

/* Batched time steps: many scenes stepped together by one captured CUDA
 * graph whose every kernel launch covers many of them (each scene runs Alg. 3
 * exactly as icr_step would; the scenes are independent problems).  At
 * creation the batch records the launch sequence of icr_step(scene, n_newton)
 * of every scene (after icr_autotune for scenes not yet tuned) and merges the
 * sequences into one common supersequence (icr_batch_merge_plan): a merged
 * launch runs one kernel for the scenes whose launch of that kernel it takes
 * over, either in one grid in which each scene's blocks see the block indices
 * of that scene's own launch, or, for kernels whose work units any grid
 * covers (assembly, CUDA-core forward-solve product, operand packing, CUDA-core
 * contraction), in one persistent grid that serves every scene's units in
 * turn.  A step of N scenes in one group makes about as many launches as the
 * longest single-scene step instead of N times as many.  Device copies and
 * fills of the step are merged the same way.  All scenes
 * must share one context, whose stream must not be the legacy default stream
 * (ICR_EINVAL), and be resident with a system, a mapping and an obstacle
 * (ICR_ESTATE); a scene may appear once.  Creation runs one batched step
 * (every scene advances one time step), then captures the graph; the launch
 * arguments (device addresses, grids) are kept in a device buffer counted
 * against the context's HBM budget (ICR_ENOMEM).  The scenes must outlive the
 * batch: icr_scene_destroy refuses a scene held by a batch (ICR_ESTATE).
 * n_groups (>= 1, at most n_scenes are used) splits the scenes into that
 * many groups balanced by cost (3 n m + 9 m^2 for n DOF and m contacts; longest
 * first, each to the least loaded group); each group's sequences are merged
 * on their own and the groups run as parallel branches of the one graph (a
 * merged launch lasts as long as its slowest scene's part, so every group
 * carries about one heavy scene, and groups overlap on the device).  Within a
 * merged launch the heaviest scene's blocks come first. */
typedef struct icr_batch icr_batch;
int icr_batch_create(icr_batch** out, icr_scene* const* scenes, int32_t n_scenes, int32_t n_newton,
                     int32_t n_groups);
/* One time step of every scene of the batch, enqueued on the context's stream
 * (the graph reads each scene's buffers, so new inputs of the same shape are
 * stepped by launching again, as with icr_step_launch).  ICR_ESTATE when a
 * scene changed since creation: evicted, a buffer reallocated, another contact
 * count, obstacle kind or parameters (create the batch again). */
int icr_batch_launch(icr_batch* batch);
typedef struct icr_batch_info_t {
  int32_t n_scenes;
  int32_t n_groups;
  int32_t launches_per_step;          /* merged launches of one batched step (kernels and copy/fill groups) */
  int32_t kernel_launches_per_step;   /* of which kernels */
  int64_t scene_launches_per_step;    /* kernel launches the scenes' own steps make together */
  uint64_t argument_bytes;            /* device buffer of the launch arguments */
  uint64_t steps;                     /* icr_batch_launch calls so far */
} icr_batch_info_t;
int icr_batch_info(icr_batch* batch, icr_batch_info_t* out);
/* One batched step run eagerly (not through the graph) with CUDA events
 * around every merged launch (diagnostic; the paper has no counterpart).
 * Synchronises; writes up to max_out entries in launch order (grouped by
 * group) and the number of merged launches to *n_out.  ICR_ESTATE when a scene
 * changed since creation, as icr_batch_launch.  name: the kernel (or
 * "copies/fills"), slots: scenes (copies and fills: operations) it covers. */
typedef struct icr_batch_launch_time {
  char name[32];
  int32_t group;
  int32_t slots;
  int32_t blocks;
  double ms;
} icr_batch_launch_time;
int icr_batch_profile(icr_batch* batch, icr_batch_launch_time* out, int32_t max_out, int32_t* n_out);
/* Waits for the context's stream, then frees the batch (not its scenes). */
int icr_batch_destroy(icr_batch* batch);
/* The merge rule of icr_batch_create on plain integer sequences (host only,
 * no GPU).  n_seq sequences of non-negative launch keys, concatenated in keys,
 * sequence i of lengths[i] keys, are merged into one common supersequence:
 * taken longest first, each sequence is aligned with the merged sequence so
 * far through a longest common subsequence of the two (shared launches where
 * both have the key in compatible order).  Writes the merged launches in
 * order: out_key[l] the key, out_count[l] how many sequences launch l covers,
 * and their indices (ascending) concatenated in out_cover, which needs room
 * for the sum of the lengths.  *n_out receives the number of merged launches
 * (ICR_EINVAL when it exceeds max_out).  Each sequence's keys are covered in
 * order, one per merged launch. */
int icr_batch_merge_plan(const int32_t* keys, const int32_t* lengths, int32_t n_seq, int32_t* out_key,
                         int32_t* out_count, int32_t* out_cover, int32_t max_out, int32_t* n_out);

/* Which paths the last icr_build_WH took, read back from the device work
 * lists (synchronises; needs icr_build_WH, ICR_ESTATE otherwise).  Diagnostic:
 * the paper has no counterpart; it shows which kernels a workload exercises. */
typedef struct icr_build_info_t {
  int32_t levels;              /* elimination-tree levels */
  int32_t tc_levels;           /* levels whose wide fronts ran the forward solve on tcgen05 */
  int32_t gemm_tc_units;       /* tensor-core front-GEMM work units (tiles x K parts) */
  int32_t gemm_tc_split_max;   /* largest K split of a level's tensor-core front GEMM (1: none split) */
  int32_t gemm_simt_units;     /* CUDA-core front-GEMM tiles */
  int32_t contract_tc_units;   /* tensor-core contraction units (tile pairs x K parts) */
  int32_t contract_tc_split;   /* K split of the tensor-core contraction (1: unsplit) */
  int32_t contract_simt_units; /* CUDA-core contraction tile pairs */
  int32_t prox_split;          /* 1: the proximity update runs as two launches (C^T lambda~ does not fit
                                  the default shared memory: 3m x element size > 48 KiB) */
  int64_t reach_nnz;           /* sum over supernodes of the contacts reaching them */
  /* algorithmic flops of the build by engine: forward solve of front s
     3q (w^2 + 2 w r) (w columns, r rows below, q reaching contacts), contraction
     w c (c + 1) with c = 3q (the upper triangle of Y_s^T Y_s) */
  double flops_front_tc, flops_front_simt, flops_contract_tc, flops_contract_simt;
  int32_t short_tile_levels;   /* levels whose CUDA-core front products use 32-row tiles */
} icr_build_info_t;
int icr_build_info(icr_scene* scene, icr_build_info_t* out);

/* Per-kernel device time (diagnostic; the paper reports per-phase times in its
 * Sec. 6 table, this splits them by kernel).  Between icr_profile_begin and
 * icr_profile_end every kernel the scene launches eagerly (not inside
 * icr_step_capture, nor a captured graph's launch) is bracketed by CUDA
 * events on the context's stream; the events serialise the launches (no
 * programmatic overlap while profiling).  icr_profile_end synchronises, then
 * writes one entry per kernel name in first-launch order: up to max_out
 * entries to out, and the number of names to *n_out. */
typedef struct icr_kernel_time {
  char name[32];
  int32_t launches;
  double total_ms;
} icr_kernel_time;
int icr_profile_begin(icr_scene* scene);
int icr_profile_end(icr_scene* scene, icr_kernel_time* out, int32_t max_out, int32_t* n_out);

/* Eviction (the paper has no counterpart: serving many scenes under an HBM
 * budget needs it).  icr_scene_evict synchronises, copies what a later time
 * step needs (the system's operators, the mapping, the obstacle, mu, the
 * gaps and directions, lambda~ and its warm start, p, p_0, u, dq) to pinned
 * host memory and frees every device byte of the scene (its buffers, the
 * input staging buffer and its captured graph), so its bytes return to the
 * context's budget.  While evicted, every other call on the scene returns
 * ICR_ESTATE.  icr_scene_readmit allocates the same buffers again
 * (ICR_ENOMEM over the budget, the scene then stays evicted), restores the
 * kept contents byte for byte and, when the scene had a captured step, captures
 * it again without running a step (the warm start is untouched); W_H and W are
 * formed again by the next step.  Evicting an evicted scene or readmitting a
 * resident one does nothing.  A device error word that was set (a timed-out
 * wait) makes icr_scene_evict return ICR_ETIMEOUT and keep the scene resident.
 * icr_scene_residency: whether the scene is resident, and the device bytes it
 * holds (or would hold again when readmitted). */
int icr_scene_evict(icr_scene* scene);
int icr_scene_readmit(icr_scene* scene);
int icr_scene_residency(icr_scene* scene, int32_t* resident, uint64_t* device_bytes);

/* Copy a field to host memory as double (float fields) or int32 (index fields).
 * `bytes` must equal the field's size; ICR_EINVAL otherwise. */
int icr_get(icr_scene* scene, int32_t field, void* dst, size_t bytes);
/* Size in bytes of a field as icr_get returns it. */
int icr_field_bytes(icr_scene* scene, int32_t field, size_t* out);
/* Number of kernels the scene has launched since it was created. */
int icr_scene_launches(icr_scene* scene, uint64_t* out);
/* Load a float field (W, LAMBDA, DELTA, C, MU, P) from host doubles, to drive
 * a single step of the path on given operands. */
int icr_set_field(icr_scene* scene, int32_t field, const double* src, size_t bytes);

/* Allocation-free elimination-tree reach (the paper has no counterpart: this
 * call exists for callers that cannot allocate device memory, such as a
 * real-time simulation or haptics loop that forbids allocation after start-up,
 * or a host framework that owns every device allocation through its own pool).
 *
 * Computes the same reach as icr_build_WH does internally: for every
 * supernode s, the ascending list of contacts whose columns of H^T reach s in
 * the supernodal elimination tree.  All pointers are DEVICE pointers owned by
 * the caller:
 *   nodes      (m x 4) int32 node ids of each contact, each in [0, n_nodes);
 *   node_super (n_nodes) int32 supernode owning each node;
 *   parent     (nsuper) int32 etree parent (> s) or -1;
 *   qcount     (nsuper) int32 output: number of contacts reaching s;
 *   qidx       (nsuper x m) int32 output: the list of supernode s starts at s*m.
 * The work is enqueued on `cuda_stream` (NULL = legacy default stream) and the
 * call returns after that stream has finished it.
 *
 * Working memory is a fixed static device array of ICR_NOALLOC_SCRATCH_WORDS
 * 32-bit words (4 MiB), held by every GPU that loads the library until the
 * process exits; the call allocates nothing.  nsuper * ceil(m / 32) must not
 * exceed that size (ICR_EINVAL otherwise).  The first call on a device looks
 * up the array's device address (cudaGetSymbolAddress) and keeps it for the
 * process, so the call must not be used across a cudaDeviceReset.  Every call
 * reads a status word back and synchronises the stream, so no call can be
 * captured into a CUDA graph: on a stream that is being captured it returns
 * ICR_ESTATE without enqueueing anything.  Every call shares the array and
 * clears the part it uses; calls that overlap on the GPU (for instance on two
 * streams) race and must be serialised by the caller.  A node id outside
 * [0, n_nodes), a supernode id outside [0, nsuper) or a parent that is neither
 * -1 nor above its child gives ICR_EINVAL with incomplete outputs. */
#define ICR_NOALLOC_SCRATCH_WORDS (1 << 20)
int icr_reach_noalloc(int32_t m, int32_t nsuper, int32_t n_nodes, const int32_t* nodes, const int32_t* node_super,
                      const int32_t* parent, int32_t* qcount, int32_t* qidx, void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* ICR_H_ */
