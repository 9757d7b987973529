/*
 * libfga -- GB300 (sm_103a) implementation of the hot path of the Fast
 * Gravitational Approach (FGA) to rigid point-set registration
 * (arXiv 2009.14005, "Fast Gravitational Approach for Rigid Point Set
 * Registration with Ordinary Differential Equations").
 *
 * Plain C ABI: host or device pointers and sizes, no C++ or framework types.
 * Notation follows the paper (Sec. IV-A): the template Y has M points and moves,
 * the reference X has N points and is fixed, D = 3.
 *
 * Conventions for every entry point
 *  - Point arrays are contiguous row-major float[n][3] (x, y, z per point),
 *    mass arrays float[n]. Unless an argument says otherwise they are DEVICE
 *    pointers on the current CUDA device, owned by the caller, and must stay
 *    valid until the work queued on `stream` has finished.
 *  - `stream` is a cudaStream_t passed as void*; NULL means the legacy default
 *    stream. Work is queued asynchronously unless the function says it
 *    synchronises.
 *  - Return value: FGA_OK (0) or a negative FGA_E* code. Nothing is thrown
 *    across the ABI. fga_last_error() returns a thread-local message for the
 *    last failure of the calling thread.
 *  - Opaque handles (fga_tree, fga_state) are owned by the library and freed by
 *    the matching *_destroy call.
 */
#ifndef FGA_H
#define FGA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ----------------------------------------------------------------- status codes */
#define FGA_OK 0
#define FGA_EINVAL -1      /* bad size, non-finite input, eps <= 0, theta < 0, ... */
#define FGA_ENOMEM -2      /* device or host allocation failed                      */
#define FGA_ECUDA -3       /* a CUDA runtime call failed (message has the name)     */
#define FGA_EDEGENERATE -4 /* a rigid fit had rank(C) < 2; best-effort R, t returned */
#define FGA_EINTERNAL -5   /* a device-side consistency check failed                */

/* ----------------------------------------------------------------- parameters */
#define FGA_DIRECT 0 /* all-pairs sum of Eq. 6                          */
#define FGA_BH 1     /* Barnes-Hut tree (Algorithm 1) + BHForce (Eq. 15) */
#define FGA_AUTO 2   /* FGA_DIRECT when N <= fga_direct_max_n(0), else FGA_BH */
#define FGA_WALK_AUTO 0 /* by template size: per-lane walks while there are too few
                           64-point groups to keep every resident warp busy,
                           else FGA_WALK_CURSOR */
#define FGA_WALK_LANE 1
#define FGA_WALK_COOP 2
#define FGA_WALK_CURSOR 3   /* one walk per 64 points that follows each point's own walk */
#define FGA_WALK_CURSOR32 4 /* the same with 32 points per warp                          */
#define FGA_WALK_CURSOR128 5 /* the same with 128 points per warp                        */

#define FGA_VEL_UNCONSTRAINED 0 /* velocities of Eq. 9 persist between iterations */
#define FGA_VEL_RIGID 1         /* velocities replaced by the rigid motion        */

#define FGA_MASS_UNIFORM 0 /* equal masses                              */
#define FGA_MASS_NIV 1     /* normalised intrinsic volume, Eq. 18       */
#define FGA_MASS_RBF 2     /* landmark RBF interpolant, Eq. 17 (fga_masses_landmarks only) */
#define FGA_MASS_SPM 3     /* smooth-particle masses, Eq. 19 (fga_masses_landmarks only)   */
#define FGA_MASS_KNN 4     /* inverse local density from the k-th nearest neighbour:
                              m_i ~ r_k(i)^D, k = `lattice` (8, 16 or 32)          */

typedef struct fga_params {
  float G;           /* gravitational constant (paper default 66.7)             */
  float eps;         /* softening length epsilon of Eq. 6 (0.2)                 */
  float eta;         /* dissipation eta of Eq. 7 (0.2)                          */
  float dt;          /* time step of Eqs. 9-10 (0.1)                            */
  float theta;       /* opening criterion of Eq. 15 (0.6)                       */
  int max_iter;      /* iterations of Algorithm 2's loop                        */
  float conv_tol;    /* stop once |T_k - T_{k-2}|_F^2 <= conv_tol; <= 0 disables */
  int method;        /* FGA_DIRECT, FGA_BH or FGA_AUTO                          */
  int normalize;     /* 1: scale inputs into [a, b] (Appendix A) in fga_register */
  float a, b;        /* normalisation range (-5, 5)                             */
  int velocity_mode; /* FGA_VEL_UNCONSTRAINED or FGA_VEL_RIGID                  */
  int max_depth;     /* BH tree depth limit, 1..20 (20)                         */
  int mass_mode;     /* reference masses in fga_register: FGA_MASS_UNIFORM, _NIV
                        or _KNN                                                */
  int lattice;       /* NIV lattice resolution varrho (16), or k for FGA_MASS_KNN */
  int profile;       /* 1: time every force-kernel launch with CUDA events on the
                        launch stream (reported in fga_stats.force_ms)           */
  int dim;           /* D: 3 (default), or 2 for planar clouds. With 2, the
                        clouds given to fga_register / fga_register_batch /
                        fga_server_submit are N x 2 and M x 2 (row-major); they
                        are registered in the plane (quadtree, 2-D NIV discs,
                        the 2 x 2 rigid fit of Eq. 14), and R_out / t_out keep
                        the 3-D layout: R = diag(R2, 1), t = (t2, ~0)         */
  int bh_walk;       /* Barnes-Hut traversal of the one-pair path (every walk
                        takes each point's own BHForce terms; the result is
                        the same up to FP32 rounding order): FGA_WALK_AUTO (0),
                        FGA_WALK_LANE (one walk per template point),
                        FGA_WALK_COOP (one walk per 64 points, each point
                        judging every node the walk visits), FGA_WALK_CURSOR /
                        FGA_WALK_CURSOR32 / FGA_WALK_CURSOR128 (one walk per
                        64 / 32 / 128 points that
                        visits the union of the points' own walks, record by
                        record)                                               */
} fga_params;

/* Fills `p` with the paper's defaults (Sec. V, parameter settings):
 * G = 66.7, eps = 0.2, eta = 0.2, dt = 0.1, theta = 0.6, [a, b] = [-5, 5],
 * depth 20, lattice 16; plus max_iter = 100, conv_tol = 0 (fixed iteration
 * count), method = FGA_BH, normalize = 1, velocity_mode = UNCONSTRAINED,
 * mass_mode = UNIFORM, profile = 0. */
void fga_params_default(fga_params* p);

typedef struct fga_stats {
  int iterations;           /* iterations actually run                         */
  int converged;            /* 1 if the conv_tol test stopped the loop         */
  int degenerate_fits;      /* iterations whose rigid fit was rank-deficient   */
  int status;               /* FGA_OK or the code that fga_register returned   */
  int64_t interactions;     /* force terms evaluated (direct: N*M per iteration;
                               BH: accepted cells + leaf particles, counted on
                               the device)                                      */
  double last_conv;         /* last |T_k - T_{k-2}|_F^2                         */
  double net_force[3];      /* sum_i m_Yi a_i of the last iteration (FP64)      */
  double torque[3];         /* sum_i (Y_i - mu_Y) x m_Yi a_i, last iteration    */
  double R_norm[9];         /* final R in the normalised frame (row-major)     */
  double t_norm[3];         /* final t in the normalised frame                  */
  double norm_info[8];      /* Xbar[3], Ybar[3], l, s of Appendix A             */
  double elapsed_ms;        /* host wall time of the call                       */
  double force_ms;          /* with profile: summed device time of the force
                               kernels (all-pairs or BH), CUDA events           */
  int force_launches;       /* with profile: number of force-kernel launches    */
  int64_t h2d_bytes;        /* fga_register: bytes copied host -> device        */
  int64_t d2h_bytes;        /* fga_register: bytes copied device -> host        */
} fga_stats;

/* ----------------------------------------------------------------- error query */
/* Message of the calling thread's last failure ("" if none). Owned by the library. */
const char* fga_last_error(void);
/* Number of kernels this library has launched in this process (all threads). */
int64_t fga_launch_count(void);

/* ----------------------------------------------------------------- Appendix A */
/* Normalisation of Appendix A, Eqs. A.1-A.3: subtracts each cloud's mean,
 * takes the global scalar minimum l and maximum r over all coordinates of both
 * centred clouds, and writes X^ = (X - Xbar - l)(b - a)/(r - l) + a (same for Y).
 * X (N x 3), Y (M x 3), Xn_out (N x 3), Yn_out (M x 3): device pointers; the
 * outputs may alias the inputs. info_out (host, 8 doubles) receives
 * {Xbar[3], Ybar[3], l, s = (b-a)/(r-l)}; the call synchronises `stream`.
 * Errors: FGA_EINVAL if N or M <= 0, b <= a, a non-finite input, or r == l. */
int fga_normalize(const float* X, int64_t N, const float* Y, int64_t M, float a, float b,
                  float* Xn_out, float* Yn_out, double info_out[8], void* stream);

/* De-normalised translation (host only, no GPU work). For a transform
 * [R | t_norm] that maps the normalised template onto the normalised
 * reference, returns t such that X = R Y + t in the original frames:
 * t = Xbar - R Ybar + l (1 - R 1) + (R a1 + t_norm - a1) / s, the solution of
 * A.3 for X (Appendix, derivation of dnorm(t)). R is row-major, unchanged by
 * the isotropic normalisation. */
void fga_denormalize(const double R[9], const double t_norm[3], const double info[8], float a,
                     double t_out[3]);

/* One rigid fit of Algorithm 2 (Eqs. 14 and 16) from reduced sums, on the
 * device, by the code every iteration of fga_step runs. With yc = y - c for a
 * template of M points y, displacements d, and the centre c = mu0 rounded to
 * FP32 (the centre the iteration kernels subtract), red (host, 27 doubles)
 * holds sum yc (3), sum d (3), S = sum yc yc^T as xx, xy, xz, yy, yz, zz (6),
 * sum d yc^T row-major (9), then 6 values the fit only copies (net force,
 * torque). The fit forms C = sum (y + d - mu_Y - mu_D)(y - mu_Y)^T, takes
 * R' = U diag(1, 1, sgn det(U V^T)) V^T of C = U S V^T (Eq. 14; R' = I when
 * sigma_2 <= 1e-7 sigma_1) and t' = mu_Y + mu_D - R' mu_Y (Eq. 16); dim = 2
 * takes the 2 x 2 fit of the x, y block. R_out (row-major 9) and t_out (3)
 * are host arrays. Synchronises `stream`. Returns FGA_EDEGENERATE for a
 * degenerate C (R' = I, t' = mu_D); FGA_EINVAL for M <= 0, dim not 2 or 3,
 * or a non-finite sum. */
int fga_rigid_fit(const double red[27], int64_t M, const double mu0[3], int dim, double R_out[9],
                  double t_out[3], void* stream);

/* ----------------------------------------------------------------- Sec. IV-F */
/* Point masses (boundary conditions, Sec. IV-F), scaled so that they sum to
 * `total`. mode = FGA_MASS_KNN: m_i ~ r_k(i)^3, r_k the distance to the k-th
 * nearest other point (k = lattice: 8, 16 or 32; n > k; r_k >= 1e-6 (b-a)).
 * mode = FGA_MASS_UNIFORM gives total/n each; FGA_MASS_NIV evaluates
 * Eq. 18 on a lattice^3 lattice over [a, b]^3 (points are expected inside the
 * normalised domain; outside points are clamped to the border cells): each
 * point carries a ball of radius (b-a)/(2*3*lattice) centred at the point
 * clamped to [a, b]^3, a cell is covered to the fraction f = V(union of its
 * points' balls, inside the cell) / V(cell) (exact along the cell's last
 * axis, where the balls cut chords on a line; midpoint rule on 64 x 64 lines
 * across it), and a point's weight is 1/f of its cell.
 * pts: device (n x 3); masses_out: device (n). lattice in 1..256.
 * Errors: FGA_EINVAL for n <= 0, bad mode/lattice, b <= a, total <= 0. */
int fga_masses(const float* pts, int64_t n, int mode, int lattice, float a, float b,
               double total, float* masses_out, void* stream);

/* Landmark-driven masses, Sec. IV-F.1 and IV-F.3.
 * mode = FGA_MASS_RBF: the RBF interpolant of Eq. 17,
 *   B(p) = sum_c lambda_c exp(-|p - p_c|^2 / sigma^2),
 * over the m landmarks p_c = pts[landmarks[c]], with lambda fixed by
 * collocation so that B = 1 at every landmark (the landmarks' strong weight;
 * an m x m FP64 Cholesky solve on the device), clamped below at `floor`
 * (> 0) so that every mass stays positive; B = 1 everywhere when m = 0.
 * mode = FGA_MASS_SPM: the smooth-particle masses of Eq. 19, S = N o B, the
 * point-wise product with the NIV weights of fga_masses (lattice, a, b).
 * The result is scaled to sum to `total`.
 * pts: device (n x 3), in the frame the masses are meant for (the
 * normalised frame for sigma in its units); landmarks: HOST array of m point
 * indices, m <= FGA_MAX_LANDMARKS; masses_out: device (n). Synchronises
 * `stream` once when m > 0.
 * Errors: FGA_EINVAL (bad sizes, modes, indices, sigma or floor <= 0,
 * repeated or coincident landmarks), FGA_ENOMEM, FGA_ECUDA. */
#define FGA_MAX_LANDMARKS 512
int fga_masses_landmarks(const float* pts, int64_t n, const int64_t* landmarks, int m, float sigma,
                         float floor, int mode, int lattice, float a, float b, double total,
                         float* masses_out, void* stream);

/* ----------------------------------------------------------------- Sec. IV-E */
typedef struct fga_tree fga_tree;

/* Barnes-Hut tree of Algorithm 1 on the (normalised) reference X with masses
 * mX: the root box is the tight bounding box of X, a cell with more than one
 * point above depth p->max_depth is split at its box midpoint into 2^3 cells
 * (points on a split plane go to the upper cell; an axis of zero extent is not
 * split), and every cell stores its diagonal l, mass and centre of mass. Cells
 * with a single non-empty child are skipped (their BH contribution equals the
 * child's). Only p->max_depth is read from `p`.
 * X: device (N x 3), mX: device (N) or NULL for masses 1/N. The tree keeps its
 * own copy of the bodies; X and mX may be freed once the stream has passed.
 * N <= 2^26 (checked before any device work).
 * Errors: FGA_EINVAL (N <= 0 or N > 2^26, bad depth, non-finite X), FGA_ENOMEM, FGA_ECUDA. */
int fga_tree_build(const float* X, const float* mX, int64_t N, const fga_params* p,
                   fga_tree** out, void* stream);
void fga_tree_destroy(fga_tree* t);
/* Number of stored cells (internal cells with >= 2 children, plus leaves). */
int64_t fga_tree_node_count(const fga_tree* t);

/* Host copy of the tree in canonical pre-order, children in octant order
 * (the same layout the FP64 oracle exports): ints (cap x 7) = depth, cell x,
 * cell y, cell z, points, is_leaf, parent; dbls (cap x 5) = mass, CoM x, y, z,
 * l; leaf_of (N, optional) = index of the leaf holding each original point.
 * Host pointers; synchronises `stream`. Returns the node count (>= 0) or an
 * FGA_E* code. Call with cap = 0 to size the buffers. */
int64_t fga_tree_export(const fga_tree* t, int64_t cap, int64_t* ints, double* dbls,
                        int64_t* leaf_of, void* stream);

/* Host copy of the records the per-point BHForce walk (Algorithm 2) reads:
 * the tree in depth-first pre-order, children in octant order, 8 floats per
 * record: CoM x, y, z, mass, l^2 (-1 for a single-particle leaf), then as
 * int32 bits the record count of the subtree (the walk's skip), the child
 * count (> 0), -1 for a single-particle leaf or -nb for a leaf with nb >= 2
 * particles, and that leaf's first particle (Morton order). A leaf with
 * nb >= 2 particles is followed by nb single-particle records, one per
 * particle. out: host, cap x 8 floats. Synchronises `stream`. Returns the
 * record count or an FGA_E* code; cap = 0 returns the count only. */
int64_t fga_tree_preorder(const fga_tree* t, int64_t cap, float* out, void* stream);

/* ----------------------------------------------------------------- Sec. IV-C/E */
/* Gravitational force on every template point, Eq. 6:
 *   F_i = G m_Yi sum_j m_Xj (X_j - Y_i) / (|X_j - Y_i|^2 + eps^2)^(3/2),
 * summed over all X (tree == NULL: X, mX, N are used) or approximated by
 * BHForce on `tree` with opening parameter p->theta (Eq. 15; X, mX, N are then
 * ignored and may be NULL). mY NULL means m_Yi = 1, i.e. the output is the
 * acceleration. FP32 arithmetic with compensated per-point accumulation;
 * with a tree, the walks' compensated sums are added exactly as 64-bit
 * fixed-point integers on a grid set by the tree's total mass and eps.
 * Y: device (M x 3); acc_out: device (M x 3), same order as Y.
 * interactions_out (host, optional): number of force terms evaluated; when
 * given, the call synchronises `stream`.
 * Errors: FGA_EINVAL (sizes, eps <= 0, theta < 0; with a tree, eps below
 * 1e-5 of the diagonal of the tree's bounding box, where that grid would no
 * longer resolve the far field to FP32 accuracy), FGA_ENOMEM, FGA_ECUDA. */
int fga_forces(const fga_tree* tree, const float* X, const float* mX, int64_t N, const float* Y,
               const float* mY, int64_t M, const fga_params* p, float* acc_out,
               int64_t* interactions_out, void* stream);

/* BHForce (Eq. 15) on `tree` as fga_forces computes it, plus the number of
 * terms each template point added (accepted cells + leaf particles of its
 * own walk, in Y's order): the per-point counterpart of interactions_out,
 * for comparing a point's walk with another implementation's. Y: device
 * (M x 3), mY: device (M) or NULL, acc_out: device (M x 3), terms_out: device
 * (M int32). Queues its work on `stream` without synchronising.
 * Errors: FGA_EINVAL (no tree, sizes, eps <= 0, theta < 0, eps below 1e-5 of
 * the diagonal of the tree's bounding box), FGA_ENOMEM, FGA_ECUDA. */
int fga_forces_terms(const fga_tree* tree, const float* Y, const float* mY, int64_t M,
                     const fga_params* p, float* acc_out, int32_t* terms_out, void* stream);

/* ----------------------------------------------------------------- no allocation */
/* Size, in float4 (16 bytes), of the device array that fga_forces_direct_static
 * uses for all its intermediate buffers: 524288 float4 = 8 MiB. */
#define FGA_STATIC_SCRATCH_FLOAT4 524288
/* float4 slots the call's state block takes at the start of that array */
#define FGA_STATIC_STATE_FLOAT4 33

/* The all-pairs forces of fga_forces(tree = NULL, ...) without any device
 * allocation. The paper has no counterpart: this entry point exists for
 * callers that must not call cudaMalloc / cudaFree, for example a loop with a
 * hard latency budget (the allocator can block and synchronise the device) or
 * a plug-in whose host application owns all device memory through its own
 * pool. Inputs, outputs and their meaning are those of fga_forces with
 * tree = NULL (X: device N x 3, mX: device N or NULL for 1/N each, Y: device
 * M x 3, mY: device M or NULL for unit masses, acc_out: device M x 3).
 * Packed inputs, per-split partial sums and the kernel's state block live in
 * one array of FGA_STATIC_SCRATCH_FLOAT4 float4 compiled into the library; it
 * occupies every device that loads the library until the process exits.
 * Limit: FGA_STATIC_STATE_FLOAT4 + N + M + 2 M <= FGA_STATIC_SCRATCH_FLOAT4,
 * i.e. 33 + N + 3 M <= 524288 (one source split; the call uses more splits
 * when they fit); larger inputs are rejected with FGA_EINVAL and a message,
 * before any GPU work. Every call looks up the array's address on the current
 * device (cudaGetSymbolAddress, which allocates nothing); the first call on a
 * device loads the library's device code there, so make it before any stream
 * capture. Every call shares
 * the array and overwrites what it reads before reading it, so leftovers of an
 * earlier call do not matter; calls that overlap on the GPU (unordered streams
 * or concurrent host threads) race on the array and must be serialised by the
 * caller. No host synchronisation. */
int fga_forces_direct_static(const float* X, const float* mX, int64_t N, const float* Y,
                             const float* mY, int64_t M, const fga_params* p, float* acc_out,
                             void* stream);

/* ----------------------------------------------------------------- Algorithm 2 */
typedef struct fga_state fga_state;

/* Device-resident state of Algorithm 2 on NORMALISED inputs with FINAL masses:
 * T = [I | 0], V = 0. Xn (N x 3), mX (N, NULL: 1/N each), Yn (M x 3),
 * mY (M, NULL: dt each, i.e. Eq. 7's friction removes the fraction eta of the
 * velocity per step) are device pointers copied into the state. For
 * p->method == FGA_BH the tree is built from Xn/mX unless `tree` is given
 * (borrowed, must outlive the state). The state keeps the template sorted
 * along a Morton curve so that neighbouring threads follow similar tree paths.
 * Errors: FGA_EINVAL (including, for FGA_BH, eps below 1e-5 of the diagonal
 * of the tree's bounding box, as in fga_forces), FGA_ENOMEM, FGA_ECUDA. */
int fga_state_create(const float* Xn, const float* mX, int64_t N, const float* Yn,
                     const float* mY, int64_t M, const fga_tree* tree, const fga_params* p,
                     fga_state** out, void* stream);

/* Queues n_iter iterations of Algorithm 2's loop body on `stream`, no host
 * synchronisation: Y = R Y0 + t; forces (Eq. 6 or BHForce); V, D (Eqs. 7-10);
 * rigid fit R', t' (Eqs. 14, 16, FP64 reduction and 3x3 SVD on the device);
 * R = R'R, t = R't + t'; convergence test. Once the test has fired, further
 * iterations are no-ops. The iterations run as one CUDA graph of force and
 * epilogue launches; an all-pairs state with N <= 4096, M <= 16384 and
 * N * M <= 2^20 runs them in one launch of one thread-block cluster instead,
 * with bit-identical results. With p->profile = 1 the launches are plain,
 * one force and one epilogue launch per iteration. Errors: FGA_EINVAL
 * (n_iter < 0), FGA_ECUDA. */
int fga_step(fga_state* s, int n_iter, void* stream);

/* Synchronises `stream` and reads the state: R (row-major, 9) and t (3) in the
 * normalised frame, and optionally stats (host). Returns FGA_EDEGENERATE if any
 * iteration's fit was rank-deficient, FGA_EINTERNAL if a device check failed. */
int fga_state_get(fga_state* s, double R[9], double t[3], fga_stats* stats, void* stream);

/* Synchronises and copies [R (9) | t (3)] after each of the first `n` iterations
 * run so far into `out` (host, n x 12). Returns the number of rows written. */
int fga_state_trajectory(fga_state* s, double* out, int n, void* stream);

void fga_state_destroy(fga_state* s);

/* Whole registration (Algorithm 2 with Appendix A): normalises X and Y into
 * [a, b] (if p->normalize), assigns masses (mX NULL: p->mass_mode with sum 1;
 * mY NULL: dt each; given masses are rescaled to those totals), builds the
 * tree for FGA_BH, runs p->max_iter iterations (fewer if conv_tol stops them)
 * and returns R, t (host, FP64) with X ~ R Y + t in the ORIGINAL frames.
 * X, Y, mX, mY may be host or device pointers (detected per pointer); host
 * inputs are copied to the device inside the call. Synchronises `stream`.
 * stats (host, optional) receives the counters and the normalised-frame result.
 * Sizes: 1 <= N, M <= 2^30; with a tree (FGA_BH, or FGA_AUTO above the
 * crossover) N <= 2^26.
 * Errors: FGA_EINVAL, FGA_ENOMEM, FGA_ECUDA, FGA_EDEGENERATE (R, t still set). */
int fga_register(const float* X, int64_t N, const float* Y, int64_t M, const float* mX,
                 const float* mY, const fga_params* p, double R_out[9], double t_out[3],
                 fga_stats* stats, void* stream);

/* ----------------------------------------------------------------- many pairs */
/* One registration problem of a batch: points and optional masses as in
 * fga_register (host or device pointers; N, M <= 2^26). */
typedef struct fga_pair {
  const float* X;
  int64_t N;
  const float* Y;
  int64_t M;
  const float* mX; /* NULL: p->mass_mode, sum 1 */
  const float* mY; /* NULL: dt each              */
  const fga_params* params; /* NULL: the call's (or server's) parameters;
                               else this pair's own (G, eps, eta, dt, theta,
                               max_iter, conv_tol, method, normalisation,
                               masses, velocity mode, max_depth), e.g. one
                               cell of a parameter grid (read during the
                               call / at submission; profile is ignored)   */
} fga_pair;

typedef struct fga_pair_result {
  double R[9], t[3];    /* X ~ R Y + t in the original frames                */
  int method;           /* FGA_DIRECT or FGA_BH, as chosen for this pair     */
  int iterations;       /* iterations run before the stop test fired (or max) */
  int converged;        /* 1 if the stop test fired                          */
  int status;           /* FGA_OK, FGA_EDEGENERATE or FGA_EINTERNAL          */
  int64_t interactions; /* force terms evaluated for this pair               */
} fga_pair_result;

/* Registers `count` independent pairs together (Algorithm 2 for each, with
 * the same parameters): every pair is normalised, given masses and, for
 * Barnes-Hut, a tree; then all pairs advance in lockstep, one iteration of
 * all pairs per force launch plus one epilogue launch (each pair's rigid fit
 * in its own block), and the p->max_iter iterations are captured in one CUDA
 * graph. With p->method == FGA_AUTO each pair takes the all-pairs sum when
 * N <= fga_direct_max_n(0) and Barnes-Hut otherwise. A pair whose stop test
 * fires (conv_tol > 0) skips the remaining work. A pair with its own
 * parameters (fga_pair.params) is registered with those: the loop runs the
 * largest max_iter of all pairs and each pair stops at its own. Results per pair go to
 * results[count] (host). stats (optional): total interactions, elapsed_ms =
 * whole call, force_ms = the iteration graph. Synchronises `stream`.
 * Errors: FGA_EINVAL (any pair invalid; message names it), FGA_ENOMEM,
 * FGA_ECUDA; FGA_EDEGENERATE / FGA_EINTERNAL if some pair reports it. */
int fga_register_batch(const fga_pair* pairs, int count, const fga_params* p,
                       fga_pair_result* results, fga_stats* stats, void* stream);

/* Crossover of FGA_AUTO: returns the current N limit for the all-pairs sum
 * and, if new_value > 0, sets it (process-wide). */
int64_t fga_direct_max_n(int64_t new_value);

/* ------------------------------------------------------------------ autotuning
 * The executors take their launch shapes and the FGA_AUTO crossover from
 * process-wide tables with built-in defaults; fga_autotune measures them on
 * this GPU (synthetic clouds generated on the device) and replaces them. */
#define FGA_TUNE_DIRECT_TILES 1 /* tile shape of the all-pairs kernel, per size class */
#define FGA_TUNE_CROSSOVER 2    /* FGA_AUTO crossover (fga_direct_max_n)              */
#define FGA_TUNE_ALL 3
#define FGA_TUNE_NSIZES 7       /* crossover probe sizes N = 1024 << k, k < 7         */

typedef struct fga_tune_report {
  int direct_bs[3], direct_qpt[3]; /* tile per template-size class: M < 8192,
                                      M < 65536, M >= 65536 (threads per block,
                                      template points per thread)             */
  double direct_gips[3];           /* G terms/s of the chosen tile (class probe) */
  int64_t direct_max_n;            /* FGA_AUTO crossover in force after the call */
  int64_t sizes[FGA_TUNE_NSIZES];  /* probed reference sizes N                  */
  double direct_us_per_point[FGA_TUNE_NSIZES]; /* all-pairs force, us per template
                                                  point and iteration            */
  double bh_us_per_point[FGA_TUNE_NSIZES];     /* Barnes-Hut force + tree build
                                                  spread over p->max_iter
                                                  iterations with M = N          */
  double bh_build_ms[FGA_TUNE_NSIZES];
  double elapsed_ms;
} fga_tune_report;

/* Measures what `flags` selects with the parameters *p (NULL: defaults; eps,
 * theta, dt and max_iter matter) and installs the result process-wide:
 * the fastest all-pairs tile for each template-size class, and the largest
 * probe N for which the all-pairs sum per template point is not slower than
 * Barnes-Hut. Takes about a second; synchronises `stream`.
 * Errors: FGA_EINVAL, FGA_ENOMEM, FGA_ECUDA. */
int fga_autotune(const fga_params* p, int flags, void* stream, fga_tune_report* out);

/* The all-pairs tile table itself: size class 0..2 as above, bs 128 or 256,
 * qpt 1, 2 or 4 (FGA_EINVAL otherwise). New states and calls use it;
 * existing states keep the plan they were created with. */
int fga_set_direct_tile(int size_class, int bs, int qpt);
int fga_get_direct_tile(int size_class, int* bs, int* qpt);

/* ------------------------------------------------------------------ serving
 * A registration server: a continuous-batching engine on one GPU. Requests
 * (pairs, Algorithm 2 with the server's parameters) are submitted at any
 * time. Admission threads (cfg->prep_threads, each with its own stream)
 * prepare each request as soon as the pair fits in the device-memory budget
 * and a slot is free (FIFO: a request waits for all requests submitted before
 * it; several are prepared at once). The prepared pair
 * (normalised template, velocities, tree or packed reference, state) stays
 * resident on the device. A runner thread advances all resident pairs
 * together, `iters_per_tick` iterations of every pair per tick (the batch
 * kernels of fga_register_batch), and between ticks adds newly prepared
 * pairs and retires the ones whose iteration limit or stop test was reached,
 * so pairs that arrive while others run join them on the device. Each pair
 * stops after exactly p->max_iter iterations (or when its stop test fires);
 * its result is the same whichever pairs it shared the device with.
 * Thread safety: submit, poll and stats may be called from any threads. */
typedef struct fga_server fga_server;

typedef struct fga_server_config {
  int64_t mem_budget;  /* device bytes resident and in-preparation pairs may hold
                          (an upper bound per pair is charged); <= 0: 3/4 of the
                          device memory free at creation                        */
  int max_pairs;       /* resident pairs at most; <= 0: 4096                      */
  int iters_per_tick;  /* iterations per tick; <= 0: 4                            */
  int device;          /* CUDA device; < 0: the calling thread's current device  */
  double max_work;     /* force terms per iteration that admitted pairs may need
                          together, estimated N*M (all-pairs) or
                          64*M*log2(N+1) (Barnes-Hut); a pair is always admitted
                          when none is held. 0: 4e9 (about 2 ms of GPU time per
                          iteration); < 0: no limit. Fewer pairs sharing the GPU
                          finish sooner; enough of them keep it busy          */
  int prep_threads;    /* threads preparing admitted requests (each with its own
                          stream; they take requests in FIFO order); <= 0: 4 */
} fga_server_config;

typedef struct fga_served {
  int64_t ticket;           /* as returned by fga_server_submit                   */
  fga_pair_result result;   /* R, t (original frames), method, iterations, ...     */
  double submit_ms;         /* host clock, ms since the server was created        */
  double admit_ms;          /* preparation started (memory and slot granted)      */
  double start_ms;          /* first tick that ran the pair                       */
  double done_ms;           /* result available to fga_server_poll                */
  char error[160];          /* message when result.status is an error, else ""    */
} fga_served;

typedef struct fga_server_stats {
  int64_t submitted, completed, failed;
  int pending;              /* waiting for admission                               */
  int preparing;            /* being prepared                                      */
  int resident;             /* on the device, iterating                            */
  int64_t bytes_charged;    /* sum of the bounds of admitted pairs                 */
  double work_admitted;     /* sum of the work estimates of admitted pairs         */
  int64_t mem_budget;
  int64_t ticks;            /* ticks run                                           */
  int64_t pair_iterations;  /* sum over ticks of resident pairs x iterations       */
  double busy_ms;           /* host time the runner spent with pairs resident      */
} fga_server_stats;

/* Creates a server with parameters *p (copied; p->method may be FGA_AUTO) and
 * configuration *cfg (NULL: all defaults). Starts its two threads.
 * Errors: FGA_EINVAL (bad parameters), FGA_ECUDA, FGA_ENOMEM. */
int fga_server_create(const fga_params* p, const fga_server_config* cfg, fga_server** out);

/* Queues one request and returns its ticket (> 0) in *ticket. req->params,
 * if set, replaces the server's parameters for this request (copied at
 * submission; max_iter >= 1). X, Y, mX, mY
 * may be host or device pointers; they are read during preparation (on the
 * server's own stream, so device data must be complete when submitted) and
 * must stay valid until the request's result has been polled. Never waits
 * for the GPU. Errors: FGA_EINVAL (null pointers, sizes outside 1..2^26, a pair
 * larger than the whole memory budget, server stopping). Bad point values
 * (NaN, zero extent) are reported in the request's result instead. */
int fga_server_submit(fga_server* srv, const fga_pair* req, int64_t* ticket);

/* Moves up to `max` finished requests (in completion order) into out[] and
 * their number into *n. If none is ready, waits up to wait_ms milliseconds
 * (0: return at once; < 0: until one is ready or nothing is outstanding). */
int fga_server_poll(fga_server* srv, fga_served* out, int max, int* n, int wait_ms);

/* Counters of the server (consistent snapshot). */
int fga_server_stats_get(fga_server* srv, fga_server_stats* out);

/* Stops the server: pending requests are dropped, the runner stops after the
 * tick it is running (pairs still resident are dropped unfinished), both
 * threads are joined and all device memory of the server is freed. Results
 * not yet polled are dropped. */
int fga_server_destroy(fga_server* srv);

#ifdef __cplusplus
}
#endif
#endif /* FGA_H */
