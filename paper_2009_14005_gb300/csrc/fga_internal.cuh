// Internal declarations shared by the libfga translation units.
// Not part of the public ABI (that is include/fga.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "fga.h"

namespace fga {

// ------------------------------------------------------------------ errors
void set_error(const std::string& msg);
void clear_error();
void count_launch(int n = 1);

struct Status {
  int code = FGA_OK;
  bool ok() const { return code == FGA_OK; }
};

#define FGA_CUDA_TRY(call)                                                          \
  do {                                                                              \
    cudaError_t _e = (call);                                                        \
    if (_e != cudaSuccess) {                                                        \
      ::fga::set_error(std::string(#call) + ": " + cudaGetErrorString(_e));         \
      return FGA_ECUDA;                                                             \
    }                                                                               \
  } while (0)

#define FGA_LAUNCH_CHECK(name)                                                      \
  do {                                                                              \
    ::fga::count_launch();                                                          \
    cudaError_t _e = cudaGetLastError();                                            \
    if (_e != cudaSuccess) {                                                        \
      ::fga::set_error(std::string("launch ") + name + ": " + cudaGetErrorString(_e)); \
      return FGA_ECUDA;                                                             \
    }                                                                               \
  } while (0)

// ------------------------------------------------------------------ memory
// Stream-ordered allocations from a library-owned pool per device (freed memory
// stays cached in the pool instead of going back to the driver).
int dev_alloc(void** p, size_t bytes, cudaStream_t s);
void dev_free(void* p, cudaStream_t s);

template <class T>
int dev_alloc_n(T** p, size_t n, cudaStream_t s) {
  return dev_alloc(reinterpret_cast<void**>(p), n * sizeof(T) + (n == 0 ? 16 : 0), s);
}

// Grid sizing: multiples of the SM count.
int sm_count();

// ------------------------------------------------------------------ device state
// Per-registration state read by the force and epilogue kernels every iteration
// and written by the rigid-fit step (the block that finishes an iteration) at
// the end of every iteration.
struct DevState {
  double R[9], t[3];      // accumulated transform, normalised frame
  double Tm1[12], Tm2[12];// [R|t] after the previous two iterations
  double mu0[3];          // centroid of the initial template
  float Rf[9], tf[3];     // FP32 copies of R, t used to place the template
  float muf[3];           // FP32 centroid of the current template, R mu0 + t
  float A[9], b[3];       // rigid-velocity coefficients: v = A y + b
  double last_conv;       // |T_k - T_{k-2}|_F^2 of the last iteration
  double netF[3], torque[3];
  unsigned long long interactions;
  int iter;               // iterations completed
  int done;               // stop: convergence, non-finite fit or iteration limit
  int converged;          // the convergence test fired
  int status;             // bit 1: non-finite fit (bit 0 unused)
  int degenerate;         // rigid fits with rank(C) < 2
  unsigned bh_next;       // BH traversal: next task slot to hand out
  unsigned bh_exited;     // BH traversal: warps that found no task left
};

// Number of FP64 reduction values per block: sum y_c (3), sum d (3),
// sum y_c y_c^T (6), sum d y_c^T (9), net force (3), torque (3).
constexpr int NRED = 27;

// ------------------------------------------------------------------ tree
// A frontier cell of the tree: the cells of the frontier partition the tree
// (every leaf lies under exactly one of them). BH work for a group of template
// points is split into one task per frontier cell. In the depth-first records
// (fga_tree::node_pre) the cell is record `node` and its subtree the records
// [node, end); path[] lists the cell's ancestors from the root (record
// indices); bit j of first_mask is set when this cell is the first frontier
// cell (in depth-first order) under path[j], i.e. the task that adds
// path[j]'s monopole for lanes that accept it.
constexpr int FRONT_MAX_PATH = 27;
struct FrontCell {
  int node;
  int npath;
  unsigned first_mask;
  int path[FRONT_MAX_PATH];
  int end;
};
#ifndef FGA_FRONT_TARGET
#define FGA_FRONT_TARGET 64
#endif
constexpr int FRONT_TARGET = FGA_FRONT_TARGET;  // frontier size the build aims for (and its cap)
// Frontier size for trees of the batch executor and the server, whose launches
// already hold many pairs' tasks: about one frontier cell per
// FGA_BATCH_FRONT_BODIES reference points, at least 8 and at most
// FRONT_TARGET (small pairs: few large tasks; large pairs: enough tasks that
// none of them decides when the launch ends).
#ifndef FGA_BATCH_FRONT_BODIES
#define FGA_BATCH_FRONT_BODIES 4096
#endif
inline int batch_front_target(int64_t N) {
  const int64_t k = (N + FGA_BATCH_FRONT_BODIES - 1) / FGA_BATCH_FRONT_BODIES;
  return (int)(k < 8 ? 8 : (k > FRONT_TARGET ? FRONT_TARGET : k));
}
}  // namespace fga

struct fga_tree {
  int64_t N = 0;          // bodies
  int64_t n_nodes = 0;    // stored cells
  int n_unique = 0;       // distinct Morton keys (= leaves)
  int max_depth = 20;
  int device = 0;
  float4* bodies = nullptr;      // N: x, y, z, m in Morton order
  int* body_index = nullptr;     // N: original index of each sorted body
  unsigned long long* keys = nullptr;  // N: sorted Morton keys
  float4* node_cm = nullptr;     // n_nodes: centre of mass xyz, mass
  int4* node_info = nullptr;     // n_nodes: {bits of l^2, first, count, depth}
                                 //  count > 0: children first .. first+count-1
                                 //  count < 0: leaf, bodies first .. first-count-1
  int2* node_bodies = nullptr;   // n_nodes: body range [x, y) of the cell
  fga::FrontCell* front = nullptr;  // frontier cells (device), depth-first order
  float4* node_pre = nullptr;    // the tree in depth-first pre-order (children in octant
                                 // order), 32 bytes per record in three arrays of n_pre
                                 // entries each (pre_cm, pre_ls, pre_cf below); a leaf with
                                 // nb >= 2 particles is followed by nb single-particle
                                 // records, one per particle
  int64_t n_pre = 0;
  int n_front = 0;
  float box_lo[3], box_hi[3];    // root box (tight bounding box of X)
  double mass_total = 0.0;       // the root cell's mass (sum of the masses of X)
  cudaStream_t stream = nullptr; // stream the buffers were allocated on
};

namespace fga {

// The depth-first records of a tree, one entry per record in each of three
// arrays (in this order in fga_tree::node_pre): CoM and mass; l^2 and the
// record count of the subtree (int bits: the walk's skip); the child count as
// in node_info and the first body of a leaf. The walks read the first two
// only: separate arrays put 8 and 16 records in a 128-byte line, so a walk's
// consecutive records share lines more often than 32-byte records would.
inline const float4* pre_cm(const fga_tree* t) { return t->node_pre; }
inline const float2* pre_ls(const fga_tree* t) {
  return reinterpret_cast<const float2*>(t->node_pre + t->n_pre);
}
inline const int2* pre_cf(const fga_tree* t) {
  return reinterpret_cast<const int2*>(pre_ls(t) + t->n_pre);
}

// ------------------------------------------------------------------ prep kernels (fga_prep.cu)
int check_finite(const float* p, int64_t n, int* d_flag, cudaStream_t s);
int check_masses(const float* m, int64_t n, int* d_flag, cudaStream_t s);
// Appendix A on the device: d_info = {Xbar[3], Ybar[3], l, s} (FP64, device),
// d_ok = 1 if r > l. Writes normalised float xyz triples.
int normalize_device(const float* X, int64_t N, const float* Y, int64_t M, float a, float b,
                     float* Xn, float* Yn, double* d_info, int* d_ok, cudaStream_t s);
int masses_device(const float* pts, int64_t n, int mode, int lattice, float a, float b,
                  double total, float* out, cudaStream_t s, int dim = 3);
// (x, y) pairs -> (x, y, 0).
int embed_planar(const float* in2, int64_t n, float* out3, cudaStream_t s);
// Rescale masses (device) so they sum to `total`.
int rescale_masses(const float* in, int64_t n, double total, float* out, cudaStream_t s);
// Tight bounding box of float xyz triples or float4 bodies (device lo/hi, 3 floats each).
int bbox_xyz(const float* p, int64_t n, float* d_lo, float* d_hi, cudaStream_t s);
// Morton keys: `bits` per axis of floor((x - lo)/(hi - lo) * 2^bits), FP64, clamped.
int morton_keys(const float* xyz, int64_t n, const float* d_lo, const float* d_hi, int bits,
                unsigned long long* keys, int* idx, cudaStream_t s);
// Stable LSD radix sort of (key, value) over the low `bits` bits; keys/vals hold
// the result, tmp buffers are scratch of the same size.
int radix_sort_pairs(unsigned long long* keys, int* vals, unsigned long long* keys_tmp,
                     int* vals_tmp, int64_t n, int bits, cudaStream_t s);
// Exclusive scan of n uint32 (device), total (device, optional).
int scan_exclusive(const unsigned* in, unsigned* out, int64_t n, unsigned* d_total,
                   cudaStream_t s);
// Centroid (FP64) of float4 xyz.
int centroid4(const float4* p, int64_t n, double* d_out3, cudaStream_t s);

// ------------------------------------------------------------------ tree (fga_tree.cu)
int tree_build(const float* X, const float* mX, int64_t N, int max_depth, fga_tree** out,
               cudaStream_t s, int front_target = FRONT_TARGET);

// ------------------------------------------------------------------ forces (fga_force.cu)
struct ForceBuffers {
  // All-pairs: S x M compensated partial sums, one slot per source split.
  float4* hi = nullptr;   // S x M (value)
  float4* lo = nullptr;   // S x M (compensation)
  int S = 1;              // number of source splits
  // Barnes-Hut: one exact fixed-point sum per point and axis, three planes of
  // M int64 (x, y, z). Every task adds its compensated FP32 sums (value and
  // compensation, each rounded to a multiple of 2^-acc_exp) with integer
  // atomics, so the result does not depend on the order of the tasks; the
  // reader (epilogue or force output) takes the value and leaves zeros for
  // the next launch. acc_exp (fixed_point_exponent) leaves every possible sum
  // of a point's terms below 2^61 units.
  long long* acc = nullptr;
  int acc_exp = 0;
};

// The binary exponent F of the Barnes-Hut fixed-point sums (value = integer
// * 2^-F). Each of a point's BHForce terms is m (s - y) / (|s - y|^2 +
// eps^2)^(3/2) for a particle or cell of mass m, whose size is at most
// m / (2.598 eps^2) (the maximum over r of r / (r^2 + eps^2)^(3/2), at r =
// eps / sqrt 2), and the terms of one point cover the reference's total mass
// once, so any partial sum is below mass_total / (2.598 eps^2) <= 2^e; F =
// 61 - e keeps it below 2^61. Clamped to [-100, 100].
int fixed_point_exponent(double mass_total, float eps);

// Plan for the all-pairs kernel: block size, queries per thread, source split.
struct DirectPlan {
  int bs = 256, qpt = 1, S = 1;
  int64_t chunk = 0;
};
DirectPlan plan_direct(int64_t N, int64_t M);
// The direct kernel's tile table (see plan_direct); size classes 0..2.
int direct_size_class(int64_t M);
bool direct_tile_supported(int bs, int qpt);
void set_direct_tile(int size_class, int bs, int qpt);
void get_direct_tile(int size_class, int* bs, int* qpt);

int launch_direct(const float4* X, int64_t N, const float4* Y0, int64_t M, const DevState* ds,
                  float eps, const DirectPlan& plan, ForceBuffers& fb, cudaStream_t s);
// kind: the walk (bh_walk_kind); order: heavy-first
// task order from launch_task_order, or null (task index order); cost: where
// each task's step count is recorded, or null; terms: per template point
// (sorted order, zeroed by the caller), the number of BHForce terms added, or null.
int launch_bh(const fga_tree* t, const float4* Y0, int64_t M, DevState* ds, float eps,
              float theta, ForceBuffers& fb, cudaStream_t s, int kind, const unsigned* order = nullptr,
              unsigned* cost = nullptr, unsigned* terms = nullptr);
// Heavy-first order of ntasks tasks from their recorded costs. `order` must
// hold ntasks + TASK_ORDER_SCRATCH entries (the tail is the sort's scratch).
constexpr unsigned TASK_ORDER_SCRATCH = 8192;

// Barnes-Hut tasks are (group of 32 * pl template points, chunk of frontier
// cells), pl points per lane (points g*32*pl + 32*q + lane, q < pl).
// bh_walk_kind(M, walk) maps fga_params.bh_walk to the kernel's walk: 0 for
// per-lane walks (pl = 1), 2 for the walk with saved sibling ranges (pl = 2),
// 3 / 4 for the union walk with two / one points per lane. FGA_WALK_AUTO
// takes the union walk with two points per lane when the template has at
// least FGA_BH_COOP_POINTS_PER_WARP points per resident warp, else per-lane
// walks: a walk for the whole warp costs fewer instructions and loads per
// point, but makes half as many tasks, each longer, and the heaviest ones (a
// group's own near field) must still spread over every warp.
#ifndef FGA_BH_COOP_POINTS_PER_WARP
#define FGA_BH_COOP_POINTS_PER_WARP 96
#endif
int bh_walk_kind(int64_t M, int walk);
inline int bh_points_per_lane(int kind) { return (kind == 0 || kind == 4) ? 1 : (kind == 5 ? 4 : 2); }
// Warps per Barnes-Hut block.
#ifndef FGA_BH_WARPS
#define FGA_BH_WARPS 4
#endif
// With FGA_BH_BLOCK_TASKS, a block takes its tasks as a whole: FGA_BH_WARPS
// adjacent groups on the same chunk, one per warp, so that the block's warps
// walk nearly the same records at the same time and share them in L1.
#ifndef FGA_BH_BLOCK_TASKS
#define FGA_BH_BLOCK_TASKS 0
#endif
// Scheduling units of a launch: (group, chunk), C chunks per group, or with
// FGA_BH_BLOCK_TASKS (block of FGA_BH_WARPS groups, chunk).
__host__ __device__ inline unsigned bh_tasks(int64_t M, int C, int pl) {
  const int64_t groups = (M + 32 * pl - 1) / (32 * pl);
  const int64_t units = FGA_BH_BLOCK_TASKS ? (groups + FGA_BH_WARPS - 1) / FGA_BH_WARPS : groups;
  return (unsigned)units * (unsigned)C;
}
// The K frontier cells are cut into C chunks of consecutive cells (chunk c:
// cells [c K / C, (c + 1) K / C)); a task walks one chunk for its group, so
// its fixed costs (the ancestor path, the conversion and atomic addition of
// its sums) are paid C times per group instead of K. C is the fewest chunks
// that still give every resident warp about
// FGA_BH_TASKS_PER_WARP tasks (0: C = K, one frontier cell per task).
#ifndef FGA_BH_TASKS_PER_WARP
#define FGA_BH_TASKS_PER_WARP 32
#endif
int bh_chunks(int64_t M, int K, int kind);
int launch_task_order(const unsigned* cost, unsigned ntasks, unsigned* order, cudaStream_t s);
// Refreshed after the first two force launches and then every
// FGA_BH_REORDER_EVERY launches (0: never, tasks run in index order).
#ifndef FGA_BH_REORDER_EVERY
#define FGA_BH_REORDER_EVERY 8
#endif
inline bool bh_reorder_due(int launches_done, int every = FGA_BH_REORDER_EVERY) {
  return every > 0 && (launches_done <= 2 || launches_done % every == 0);
}
// The same schedule for the batch executor and the server.
#ifndef FGA_BATCH_REORDER_EVERY
#define FGA_BATCH_REORDER_EVERY 8
#endif

struct EpiParams {
  float G, dt, eta;
  int vmode;
  double conv_tol;
  int max_traj;
  double inv_M, inv_dt;  // 1/M and 1/dt, FP64, computed on the host
  int max_iter;          // > 0: the pair stops by itself after this many iterations
  int dim;               // 2: planar clouds, the 2 x 2 rigid fit; otherwise 3-D
};
int launch_epilogue(const float4* Y0, int64_t M, const ForceBuffers& fb, float4* V,
                    DevState* ds, double* d_partials, unsigned* d_counter, double* d_traj,
                    const EpiParams& ep, cudaStream_t s, unsigned long long inter_add);
int epilogue_blocks(int64_t M);
// acc_out[perm[i]] = G * mY[i] * sum of partials (or the acceleration if mY is null).
int launch_forces_out(const ForceBuffers& fb, int64_t M, const float4* Y0, int use_mass,
                      float G, const int* perm, float* acc_out, cudaStream_t s);
// The whole iteration loop of a small all-pairs pair in one launch of one
// thread-block cluster (fga_small.cu), bit-identical to the separate force
// and epilogue launches. Eligible: N <= FGA_SMALL_LOOP_MAX_N (the sources are
// staged in shared memory), M <= FGA_SMALL_LOOP_MAX_M and N * M <=
// FGA_SMALL_LOOP_MAX_TERMS (beyond that the full GPU's separate launches are
// faster than one cluster's SMs); available: the device holds a cluster of
// the kernel (checked once per device and tile shape).
#ifndef FGA_SMALL_LOOP_MAX_N
#define FGA_SMALL_LOOP_MAX_N 4096
#endif
#ifndef FGA_SMALL_LOOP_MAX_M
#define FGA_SMALL_LOOP_MAX_M 16384
#endif
#ifndef FGA_SMALL_LOOP_MAX_TERMS
#define FGA_SMALL_LOOP_MAX_TERMS (1 << 20)
#endif
bool small_loop_eligible(int64_t N, int64_t M, const DirectPlan& plan);
bool small_loop_available(const DirectPlan& plan);
// n_iter iterations; the trajectory is written for the first traj_iters.
int launch_small_loop(const float4* X4, int64_t N, const float4* Y0, int64_t M, DevState* ds, float eps,
                      const DirectPlan& plan, const ForceBuffers& fb, float4* V, double* partials,
                      double* traj, int traj_iters, const EpiParams& ep, unsigned long long inter_add,
                      int n_iter, cudaStream_t s);
// Initialise DevState (identity transform, mu0 from d_mu0).
int launch_state_init(DevState* ds, const double* d_mu0, cudaStream_t s);

// Scope guard for temporary device buffers of one call.
struct Scratch {
  cudaStream_t s;
  std::vector<void*> ptrs;
  explicit Scratch(cudaStream_t st) : s(st) {}
  ~Scratch() {
    for (void* p : ptrs) dev_free(p, s);
  }
  template <class T>
  int alloc(T** p, size_t n) {
    int rc = dev_alloc_n(p, n, s);
    if (rc == FGA_OK) ptrs.push_back(*p);
    return rc;
  }
};


// Host helpers of fga_api.cu shared with the batch executor.
int check_params(const fga_params* p, bool need_tree);
int check_register_params(const fga_params* p);
// FGA_AUTO -> FGA_DIRECT or FGA_BH by the reference size (fga_batch.cu).
int resolve_method(const fga_params* p, int64_t N);
int read_flags(const int* d_flags, int n, int* h, cudaStream_t s);
unsigned grid_for(int64_t n);
bool is_device_ptr(const void* p);
int pack_template(const float* Y, const float* mY, float m_default, int64_t M, bool sort,
                  float4* Y0, int* perm, cudaStream_t s);
struct Prepared {
  float *Xn = nullptr, *Yn = nullptr, *mXn = nullptr, *mYn = nullptr;
  double* info = nullptr;
  int* flags = nullptr;
};
int prepare_inputs(Scratch& sc, const float* X, int64_t N, const float* Y, int64_t M,
                   const float* mX, const float* mY, const fga_params* p, Prepared& out,
                   int64_t& h2d, cudaStream_t s);


}  // namespace fga
